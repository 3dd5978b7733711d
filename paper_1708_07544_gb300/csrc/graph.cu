// Connection graph of a determinant space and the FP64 sigma H c.
//
// Sec. IV: every single and double excitation between pairs of determinants
// of V is generated to evaluate the Hamiltonian.  Instead of generating the
// ~N^2 n^2 excitations of each row and looking them up, the determinants are
// grouped by alpha string (V is sorted by (alpha, beta)) and by beta string
// (a second, beta-major order), and connections are found by XOR/popcount
// scans:
//   (A) same alpha string, beta differs by 1 or 2 electrons;
//   (B) same beta string, alpha differs by 1 or 2 electrons;
//   (C) alpha differs by a single (via the single-excitation neighbours of
//       each distinct alpha string) and beta differs by a single.
// The three sets are disjoint.  Rows are filled in scan order, so the CSR
// layout (and the sigma summation order) is deterministic.
#include "hci_internal.cuh"

namespace {

constexpr int G_WARPS = 8;

__device__ __forceinline__ bool key_less(ulonglong2 a, ulonglong2 b) {
  return a.x < b.x || (a.x == b.x && a.y < b.y);
}
__device__ __forceinline__ int64_t lower_bound_k(const ulonglong2* __restrict__ arr, int64_t n, ulonglong2 key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (key_less(arr[mid], key)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int64_t lower_bound_u(const uint64_t* __restrict__ arr, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (arr[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// grouping
// ---------------------------------------------------------------------------
// word = 0: group by .x (alpha) of keys; word = 1: by .x of swapped keys
__global__ void k_run_flags(const ulonglong2* __restrict__ keys, int64_t n, int64_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || keys[i].x != keys[i - 1].x) ? 1 : 0;
}

// group index per element, unique strings and group starts
__global__ void k_groups(const ulonglong2* __restrict__ keys, int64_t n, const int64_t* __restrict__ flag,
                         const int64_t* __restrict__ excl, int32_t* __restrict__ gidx, uint64_t* __restrict__ uniq,
                         int64_t* __restrict__ start) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t g = excl[i] + flag[i] - 1;
    gidx[i] = (int32_t)g;
    if (flag[i]) {
      uniq[g] = keys[i].x;
      start[g] = i;
    }
  }
}

__global__ void k_set_last(int64_t* start, const int64_t* ngroups_dev, int64_t n) {
  start[*ngroups_dev] = n;
}

__global__ void k_store_at(int64_t* arr, int64_t idx, const int64_t* val) { arr[idx] = *val; }

__global__ void k_swap_keys(const ulonglong2* __restrict__ in, int64_t n, ulonglong2* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 k = in[i];
    out[i] = make_ulonglong2(k.y, k.x);
  }
}

// permb[k] = index in V of the k-th determinant in beta-major order;
// ib[permb[k]] = beta group of position k
__global__ void k_perm_b(const ulonglong2* __restrict__ bkeys, int64_t n, const ulonglong2* __restrict__ V,
                         const int32_t* __restrict__ bgroup_of_pos, int32_t* __restrict__ permb,
                         int32_t* __restrict__ ib) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 s = bkeys[k];
    int64_t j = lower_bound_k(V, n, make_ulonglong2(s.y, s.x));
    permb[k] = (int32_t)j;
    ib[j] = bgroup_of_pos[k];
  }
}

// single-excitation neighbours (within the distinct alpha strings) of each
// distinct alpha string; count pass (out == nullptr) or fill pass
__global__ void k_alpha_nbrs(int n, const uint64_t* __restrict__ ua, int64_t nua, const int64_t* __restrict__ ptr,
                             int64_t* __restrict__ cnt, int32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = warp; g < nua; g += nwarps) {
    uint64_t s = ua[g];
    int64_t w = out ? ptr[g] : 0;
    int64_t c = 0;
    const int npairs = n * n;
    for (int b0 = 0; b0 < npairs; b0 += 32) {
      int t = b0 + lane;
      bool hit = false;
      int64_t idx = -1;
      if (t < npairs) {
        int p = t / n, r = t % n;
        if (((s >> p) & 1ull) && !((s >> r) & 1ull)) {
          uint64_t x = s ^ (1ull << p) ^ (1ull << r);
          int64_t pos = lower_bound_u(ua, nua, x);
          if (pos < nua && ua[pos] == x) { hit = true; idx = pos; }
        }
      }
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (out && hit) out[w + c + __popc(m & ((1u << lane) - 1u))] = (int32_t)idx;
      c += __popc(m);
    }
    if (!out && lane == 0) cnt[g] = c;
  }
}

// ---------------------------------------------------------------------------
// Slater-Condon element <D_i|H|D_j> for a known connection
// ---------------------------------------------------------------------------
struct HamView {
  int n;
  const double* h;
  const double* eri;
  const double* jk_same;
  const double* j_opp;
};

__device__ __forceinline__ double eri4(const HamView& H, int p, int q, int r, int s) {
  return H.eri[(((int64_t)p * H.n + q) * H.n + r) * H.n + s];
}

// single p->r in spin string sj (other spin string oj), both of D_j
__device__ __forceinline__ double single_el(const HamView& H, uint64_t sj, uint64_t oj, int p, int r) {
  double v = H.h[p * H.n + r];
  const double* js = H.jk_same + ((int64_t)p * H.n + r) * H.n;
  const double* jo = H.j_opp + ((int64_t)p * H.n + r) * H.n;
  for (int k = 0; k < H.n; ++k) {
    if ((sj >> k) & 1ull) v += js[k];
    if ((oj >> k) & 1ull) v += jo[k];
  }
  return exc_phase(sj, p, r) * v;
}

__device__ __forceinline__ double same_double_el(const HamView& H, uint64_t sj, uint64_t x) {
  uint64_t holes = sj & x, parts = x & ~sj;
  int p = __ffsll((long long)holes) - 1; holes &= holes - 1;
  int q = __ffsll((long long)holes) - 1;
  int r = __ffsll((long long)parts) - 1; parts &= parts - 1;
  int s = __ffsll((long long)parts) - 1;
  double s1 = exc_phase(sj, p, r);
  uint64_t t = sj ^ (1ull << p) ^ (1ull << r);
  double s2 = exc_phase(t, q, s);
  return s1 * s2 * (eri4(H, p, r, q, s) - eri4(H, p, s, q, r));
}

__device__ double connection_el(const HamView& H, ulonglong2 ki, ulonglong2 kj) {
  uint64_t xa = ki.x ^ kj.x, xb = ki.y ^ kj.y;
  int da = __popcll(xa), db = __popcll(xb);
  if (da == 0) {
    if (db == 2) {
      int p = __ffsll((long long)(kj.y & xb)) - 1, r = __ffsll((long long)(ki.y & xb)) - 1;
      return single_el(H, kj.y, kj.x, p, r);
    }
    return same_double_el(H, kj.y, xb);
  }
  if (db == 0) {
    if (da == 2) {
      int p = __ffsll((long long)(kj.x & xa)) - 1, r = __ffsll((long long)(ki.x & xa)) - 1;
      return single_el(H, kj.x, kj.y, p, r);
    }
    return same_double_el(H, kj.x, xa);
  }
  int p = __ffsll((long long)(kj.x & xa)) - 1, r = __ffsll((long long)(ki.x & xa)) - 1;
  int q = __ffsll((long long)(kj.y & xb)) - 1, s = __ffsll((long long)(ki.y & xb)) - 1;
  return exc_phase(kj.x, p, r) * exc_phase(kj.y, q, s) * eri4(H, p, r, q, s);
}

// ---------------------------------------------------------------------------
// row traversal: (A) alpha group, (B) beta group, (C) alpha-single x beta-single
// ---------------------------------------------------------------------------
struct GraphArgs {
  const ulonglong2* V;
  int64_t nV;
  const int32_t* ia;       // alpha group of each det
  const int64_t* ga;       // alpha group starts [nua+1]
  const int32_t* ib;       // beta group of each det
  const int64_t* gb;       // beta group starts (beta-major positions) [nub+1]
  const int32_t* permb;    // beta-major position -> det
  const int64_t* nbr_ptr;  // alpha single neighbours
  const int32_t* nbr;
  const int64_t* rowptr;   // fill pass
  int32_t* col;
  double* val;
  int64_t* rowcnt;         // count pass
  unsigned long long* queue;
  HamView H;
};

template <bool FILL>
__device__ __forceinline__ void visit(const GraphArgs& A, int64_t i, ulonglong2 ki, int64_t j, bool ok, int64_t& w) {
  const int lane = threadIdx.x & 31;
  unsigned m = __ballot_sync(0xffffffffu, ok);
  if (FILL && ok) {
    int64_t pos = w + __popc(m & ((1u << lane) - 1u));
    A.col[pos] = (int32_t)j;
    A.val[pos] = connection_el(A.H, ki, A.V[j]);
  }
  w += __popc(m);
}

template <bool FILL>
__global__ void __launch_bounds__(G_WARPS * 32) k_rows(GraphArgs A) {
  __shared__ int64_t s_start[G_WARPS][32];
  __shared__ int64_t s_pref[G_WARPS][33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  while (true) {
    unsigned long long qi = 0;
    if (lane == 0) qi = atomicAdd(A.queue, 1ull);
    const int64_t i = (int64_t)__shfl_sync(0xffffffffu, qi, 0);
    if (i >= A.nV) break;
    const ulonglong2 ki = A.V[i];
    int64_t w = FILL ? A.rowptr[i] : 0;
    // (A) same alpha string
    {
      int g = A.ia[i];
      int64_t b = A.ga[g], e = A.ga[g + 1];
      for (int64_t j0 = b; j0 < e; j0 += 32) {
        int64_t j = j0 + lane;
        bool ok = false;
        if (j < e && j != i) {
          int d = __popcll(ki.y ^ A.V[j].y);
          ok = d == 2 || d == 4;
        }
        visit<FILL>(A, i, ki, j, ok, w);
      }
    }
    // (B) same beta string
    {
      int g = A.ib[i];
      int64_t b = A.gb[g], e = A.gb[g + 1];
      for (int64_t k0 = b; k0 < e; k0 += 32) {
        int64_t k = k0 + lane;
        bool ok = false;
        int64_t j = -1;
        if (k < e) {
          j = A.permb[k];
          if (j != i) {
            int d = __popcll(ki.x ^ A.V[j].x);
            ok = d == 2 || d == 4;
          }
        }
        visit<FILL>(A, i, ki, j, ok, w);
      }
    }
    // (C) alpha single neighbours, beta single: flattened over the
    // concatenation of the neighbour groups, 32 groups at a time
    {
      int g = A.ia[i];
      int64_t nb0 = A.nbr_ptr[g], nb1 = A.nbr_ptr[g + 1];
      for (int64_t c0 = nb0; c0 < nb1; c0 += 32) {
        int64_t cidx = c0 + lane;
        int64_t st = 0, sz = 0;
        if (cidx < nb1) {
          int gg = A.nbr[cidx];
          st = A.ga[gg];
          sz = A.ga[gg + 1] - st;
        }
        // inclusive scan of sizes
        int64_t inc = sz;
        for (int o = 1; o < 32; o <<= 1) {
          int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += t;
        }
        s_start[wid][lane] = st;
        s_pref[wid][lane + 1] = inc;
        if (lane == 0) s_pref[wid][0] = 0;
        __syncwarp();
        const int64_t total = s_pref[wid][32];
        for (int64_t v0 = 0; v0 < total; v0 += 32) {
          int64_t v = v0 + lane;
          bool ok = false;
          int64_t j = -1;
          if (v < total) {
            int lo = 0, hi = 31;     // find group t with pref[t] <= v < pref[t+1]
            while (lo < hi) {
              int mid = (lo + hi + 1) >> 1;
              if (s_pref[wid][mid] <= v) lo = mid;
              else hi = mid - 1;
            }
            j = s_start[wid][lo] + (v - s_pref[wid][lo]);
            ok = __popcll(ki.y ^ A.V[j].y) == 2;
          }
          visit<FILL>(A, i, ki, j, ok, w);
        }
        __syncwarp();
      }
    }
    if (!FILL && lane == 0) A.rowcnt[i] = w;
  }
}

// diagonal <D|H|D> (includes e_core)
__global__ void k_diag(int n, const double* __restrict__ h, const double* __restrict__ eri, double ecore,
                       const ulonglong2* __restrict__ V, int64_t nV, double* __restrict__ out) {
  extern __shared__ double sm[];
  double* J = sm;            // (kk|ll)
  double* K = sm + n * n;    // (kl|lk)
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int k = t / n, l = t % n;
    J[t] = eri[(((int64_t)k * n + k) * n + l) * n + l];
    K[t] = eri[(((int64_t)k * n + l) * n + l) * n + k];
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 key = V[i];
    double e1 = 0.0, e2 = 0.0;
    for (int s = 0; s < 2; ++s) {
      uint64_t x = s == 0 ? key.x : key.y;
      uint64_t o = s == 0 ? key.y : key.x;
      uint64_t a = x;
      while (a) {
        int k = __ffsll((long long)a) - 1;
        a &= a - 1;
        e1 += h[k * n + k];
        // same spin pairs l > k, opposite spin pairs counted once (s == 0)
        uint64_t b = x & ~((2ull << k) - 1ull);
        while (b) {
          int l = __ffsll((long long)b) - 1;
          b &= b - 1;
          e2 += J[k * n + l] - K[k * n + l];
        }
        if (s == 0) {
          uint64_t c = o;
          while (c) {
            int l = __ffsll((long long)c) - 1;
            c &= c - 1;
            e2 += J[k * n + l];
          }
        }
      }
    }
    out[i] = ecore + e1 + e2;
  }
}

// sigma = diag .* c + offdiag * c ; one warp per row, nvec vectors
__global__ void __launch_bounds__(256) k_sigma(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                               const double* __restrict__ val, const double* __restrict__ diag,
                                               int64_t nV, const double* __restrict__ c, double* __restrict__ sigma,
                                               int nvec) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < nV; i += nwarps) {
    const int64_t b = rowptr[i], e = rowptr[i + 1];
    for (int v0 = 0; v0 < nvec; v0 += 4) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      const int nv = nvec - v0 < 4 ? nvec - v0 : 4;
      for (int64_t k = b + lane; k < e; k += 32) {
        const int64_t j = col[k];
        const double hv = val[k];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < nv) acc[t] = fma(hv, c[(int64_t)(v0 + t) * nV + j], acc[t]);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        double a = acc[t];
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        acc[t] = a;
      }
      if (lane < nv) {
        double a = lane == 0 ? acc[0] : lane == 1 ? acc[1] : lane == 2 ? acc[2] : acc[3];
        const int64_t o = (int64_t)(v0 + lane) * nV + i;
        sigma[o] = fma(diag[i], c[o], a);
      }
    }
  }
}

}  // namespace

hci_status graph_build(hci_ctx* ctx, const uint64_t* keys, int64_t nV) {
  Graph& G = ctx->graph;
  G.valid = false;
  const int n = ctx->n;
  const ulonglong2* V = reinterpret_cast<const ulonglong2*>(keys);
  if (nV >= ((int64_t)1 << 31) - 1) return hci_fail(ctx, HCI_ERR_INVALID, "graph: nV exceeds int32 columns");
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  int64_t* dtot = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 40);
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(bp<char>(ctx->s_counter) + 48);
  // keep a private copy of the keys (the caller's buffer may change)
  HCI_TRY(ensure_buf(ctx, G.keys, (size_t)nV * 16));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.keys.p, keys, (size_t)nV * 16, cudaMemcpyDeviceToDevice, ctx->st));
  V = bp<ulonglong2>(G.keys);
  // --- alpha groups
  HCI_TRY(ensure_buf(ctx, ctx->s_flags, (size_t)(2 * nV + 1) * 8));
  int64_t* flag = bp<int64_t>(ctx->s_flags);
  int64_t* excl = flag + nV;
  HCI_TRY(ensure_buf(ctx, ctx->g_ia, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, ctx->g_ua, (size_t)nV * 8));
  HCI_TRY(ensure_buf(ctx, ctx->g_ga, (size_t)(nV + 1) * 8));
  const int gb = grid_for(nV, 256);
  k_run_flags<<<gb, 256, 0, ctx->st>>>(V, nV, flag);
  HCI_TRY(scan_i64(ctx, flag, excl, nV, dtot));
  k_groups<<<gb, 256, 0, ctx->st>>>(V, nV, flag, excl, bp<int32_t>(ctx->g_ia), bp<uint64_t>(ctx->g_ua),
                                     bp<int64_t>(ctx->g_ga));
  k_set_last<<<1, 1, 0, ctx->st>>>(bp<int64_t>(ctx->g_ga), dtot, nV);
  int64_t nua = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&nua, dtot, 8, cudaMemcpyDeviceToHost, ctx->st));
  // --- beta-major order and beta groups
  HCI_TRY(ensure_buf(ctx, ctx->g_bkeys, (size_t)nV * 16));
  HCI_TRY(ensure_buf(ctx, ctx->g_bkeys2, (size_t)nV * 16));
  k_swap_keys<<<gb, 256, 0, ctx->st>>>(V, nV, bp<ulonglong2>(ctx->g_bkeys));
  HCI_TRY(sort_keys(ctx, bp<uint64_t>(ctx->g_bkeys), bp<uint64_t>(ctx->g_bkeys2), nV, n, n));
  HCI_TRY(ensure_buf(ctx, ctx->g_ub, (size_t)nV * 8));
  HCI_TRY(ensure_buf(ctx, ctx->g_gb, (size_t)(nV + 1) * 8));
  HCI_TRY(ensure_buf(ctx, ctx->g_ib, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, ctx->g_permb, (size_t)nV * 4));
  // reuse bkeys2 (now scratch) as int32 group-of-position
  int32_t* bgroup_of_pos = bp<int32_t>(ctx->g_bkeys2);
  k_run_flags<<<gb, 256, 0, ctx->st>>>(bp<ulonglong2>(ctx->g_bkeys), nV, flag);
  HCI_TRY(scan_i64(ctx, flag, excl, nV, dtot));
  k_groups<<<gb, 256, 0, ctx->st>>>(bp<ulonglong2>(ctx->g_bkeys), nV, flag, excl, bgroup_of_pos,
                                     bp<uint64_t>(ctx->g_ub), bp<int64_t>(ctx->g_gb));
  k_set_last<<<1, 1, 0, ctx->st>>>(bp<int64_t>(ctx->g_gb), dtot, nV);
  k_perm_b<<<gb, 256, 0, ctx->st>>>(bp<ulonglong2>(ctx->g_bkeys), nV, V, bgroup_of_pos, bp<int32_t>(ctx->g_permb),
                                     bp<int32_t>(ctx->g_ib));
  HCI_CUDA(ctx, cudaGetLastError());
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  // --- alpha single neighbours
  HCI_TRY(ensure_buf(ctx, ctx->g_cnt, (size_t)(nua + 1) * 8));
  HCI_TRY(ensure_buf(ctx, ctx->g_nbr_ptr, (size_t)(nua + 1) * 8));
  const int gw = grid_for(nua * 32, 256);
  k_alpha_nbrs<<<gw, 256, 0, ctx->st>>>(n, bp<uint64_t>(ctx->g_ua), nua, nullptr, bp<int64_t>(ctx->g_cnt), nullptr);
  HCI_TRY(scan_i64(ctx, bp<int64_t>(ctx->g_cnt), bp<int64_t>(ctx->g_nbr_ptr), nua, dtot));
  k_store_at<<<1, 1, 0, ctx->st>>>(bp<int64_t>(ctx->g_nbr_ptr), nua, dtot);
  int64_t nnbr = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&nnbr, dtot, 8, cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  HCI_TRY(ensure_buf(ctx, ctx->g_nbr, (size_t)(nnbr + 1) * 4));
  k_alpha_nbrs<<<gw, 256, 0, ctx->st>>>(n, bp<uint64_t>(ctx->g_ua), nua, bp<int64_t>(ctx->g_nbr_ptr), nullptr,
                                         bp<int32_t>(ctx->g_nbr));
  HCI_CUDA(ctx, cudaGetLastError());
  // --- count pass
  GraphArgs A;
  A.V = V; A.nV = nV;
  A.ia = bp<int32_t>(ctx->g_ia); A.ga = bp<int64_t>(ctx->g_ga);
  A.ib = bp<int32_t>(ctx->g_ib); A.gb = bp<int64_t>(ctx->g_gb);
  A.permb = bp<int32_t>(ctx->g_permb);
  A.nbr_ptr = bp<int64_t>(ctx->g_nbr_ptr); A.nbr = bp<int32_t>(ctx->g_nbr);
  A.H = HamView{n, bp<double>(ctx->h), bp<double>(ctx->eri), bp<double>(ctx->jk_same), bp<double>(ctx->j_opp)};
  A.queue = queue;
  HCI_TRY(ensure_buf(ctx, G.rowptr, (size_t)(nV + 1) * 8));
  A.rowcnt = flag;   // reuse
  A.rowptr = nullptr; A.col = nullptr; A.val = nullptr;
  const int grows = 152 * 8;
  HCI_CUDA(ctx, cudaMemsetAsync(queue, 0, 8, ctx->st));
  k_rows<false><<<grows, G_WARPS * 32, 0, ctx->st>>>(A);
  HCI_CUDA(ctx, cudaGetLastError());
  HCI_TRY(scan_i64(ctx, flag, bp<int64_t>(G.rowptr), nV, dtot));
  k_store_at<<<1, 1, 0, ctx->st>>>(bp<int64_t>(G.rowptr), nV, dtot);
  int64_t nnz = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&nnz, dtot, 8, cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  // --- fill pass
  HCI_TRY(ensure_buf(ctx, G.col, (size_t)(nnz + 1) * 4));
  HCI_TRY(ensure_buf(ctx, G.val, (size_t)(nnz + 1) * 8));
  A.rowptr = bp<int64_t>(G.rowptr); A.col = bp<int32_t>(G.col); A.val = bp<double>(G.val);
  A.rowcnt = nullptr;
  HCI_CUDA(ctx, cudaMemsetAsync(queue, 0, 8, ctx->st));
  k_rows<true><<<grows, G_WARPS * 32, 0, ctx->st>>>(A);
  HCI_CUDA(ctx, cudaGetLastError());
  // --- diagonal
  HCI_TRY(ensure_buf(ctx, G.diag, (size_t)nV * 8));
  HCI_CUDA(ctx, cudaFuncSetAttribute(k_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 8));
  k_diag<<<grid_for(nV, 128), 128, (size_t)2 * n * n * 8, ctx->st>>>(n, bp<double>(ctx->h), bp<double>(ctx->eri),
                                                                     ctx->ecore, V, nV, bp<double>(G.diag));
  HCI_CUDA(ctx, cudaGetLastError());
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  G.nV = nV;
  G.nnz = nnz;
  G.valid = true;
  return HCI_OK;
}

hci_status graph_ensure(hci_ctx* ctx, const uint64_t* keys, int64_t nV) {
  uint64_t hsh = 0;
  HCI_TRY(hash_keys(ctx, keys, nV, &hsh));
  if (ctx->graph.valid && ctx->graph.nV == nV && ctx->graph.hash == hsh) return HCI_OK;
  int ok = 0;
  HCI_TRY(check_sorted(ctx, keys, nV, &ok));
  if (!ok) return hci_fail(ctx, HCI_ERR_INVALID, "keys are not strictly ascending");
  HCI_TRY(graph_build(ctx, keys, nV));
  ctx->graph.hash = hsh;
  return HCI_OK;
}

hci_status sigma_apply(hci_ctx* ctx, const double* c, double* sigma, int nvec) {
  Graph& G = ctx->graph;
  k_sigma<<<grid_for(G.nV * 32, 256, 152 * 16), 256, 0, ctx->st>>>(
      bp<int64_t>(G.rowptr), bp<int32_t>(G.col), bp<double>(G.val), bp<double>(G.diag), G.nV, c, sigma, nvec);
  HCI_CUDA(ctx, cudaGetLastError());
  return HCI_OK;
}

extern "C" hci_status hci_sigma(hci_ctx* ctx, const uint64_t* keys, int64_t nV, const double* c, double* sigma,
                                int nvec) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_sigma: null context");
  if (nV <= 0 || nvec <= 0) return hci_fail(ctx, HCI_ERR_INVALID, "hci_sigma: empty space or no vectors");
  if (!keys || !c || !sigma) return hci_fail(ctx, HCI_ERR_INVALID, "hci_sigma: null pointer");
  HCI_TRY(graph_ensure(ctx, keys, nV));
  return sigma_apply(ctx, c, sigma, nvec);
}
