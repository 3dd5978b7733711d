// Selection step of variational HCI (Sec. II.A, Eq. criteria, Fig. 1b):
// heat-bath walk over the sorted double-excitation lists, exact singles
// behind an upper-bound screen, sort-based deduplication against V, and the
// sorted merge V^{mu+1} = V^mu + C^mu.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hci_internal.cuh"

namespace {

constexpr int SEL_WARPS = 8;          // warps per CTA in the walk kernels
constexpr int WALK_CHUNK = 256;       // list entries per walk work item

struct WalkArgs {
  int n, na, nb;
  const ulonglong2* keys;
  const double* c;
  int64_t nV;
  double eps1;
  int accept_all;
  const double* opp_mag;
  const uint16_t* opp_tgt;
  int Lo;
  const double* same_mag;
  const uint16_t* same_tgt;
  int Ls;
  double max_dbl;        // largest magnitude in any list
  const double* list_max; // [n*n] opposite-spin then [n(n-1)/2] same-spin list maxima
  const double* h;
  const double* jk_same;
  const double* j_opp;
  const double* single_bound;
  double max_single;
  ulonglong2* out;
  int64_t cap;
  unsigned long long* counter;     // [0] candidates, [1] next det (work queue)
  unsigned long long* walkstat;    // [0] list entries walked, [1] exact singles
  int4* items;                     // walk work items {det, code, start, end}
  int64_t item_cap;
  unsigned long long* nitems;
  const double* f_ref;             // [2][n][n] single-excitation rows of the aufbau determinant
  uint64_t ref_a, ref_b;
  // perturbative mode (vals != nullptr): every emitted target also gets its
  // term H_ai c_i, emitted only when |H_ai c_i| > eps1 and the target's hash
  // class is `part` of `npart`
  double* vals;
  int32_t* srcs;         // perturbative mode with sources: source determinant of each pair; vals then
                         // holds the element H_ai instead of the term H_ai c_i
  int npart, part;
  const double* eri;
};

__device__ __forceinline__ uint64_t key_mix(ulonglong2 k) {
  uint64_t x = k.x * 0x9E3779B97F4A7C15ull ^ (k.y + 0x632BE59BD9B4E019ull + (k.x << 6) + (k.x >> 2));
  x ^= x >> 31; x *= 0xBF58476D1CE4E5B9ull; x ^= x >> 29;
  return x;
}

// perturbative mode: keep the term and the target?
__device__ __forceinline__ bool pt_keep(const WalkArgs& A, ulonglong2 key, double term) {
  return fabs(term) > A.eps1 && (A.npart <= 1 || (int)(key_mix(key) % (uint64_t)A.npart) == A.part);
}

__device__ __forceinline__ void tri_decode_dev(int t, int& lo, int& hi) {
  int h = (int)((1.0 + sqrt(1.0 + 8.0 * (double)t)) * 0.5);
  while (h * (h - 1) / 2 > t) --h;
  while ((h + 1) * h / 2 <= t) ++h;
  hi = h;
  lo = t - h * (h - 1) / 2;
}

// Warp-aggregated append of one optional key (and term) per lane.
__device__ __forceinline__ void warp_emit(bool emit, ulonglong2 key, double term, int src, const WalkArgs& A) {
  const int lane = threadIdx.x & 31;
  unsigned m = __ballot_sync(0xffffffffu, emit);
  if (!m) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&A.counter[0], (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (emit) {
    unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
    if ((int64_t)idx < A.cap) {
      A.out[idx] = key;
      if (A.vals) A.vals[idx] = term;
      if (A.srcs) A.srcs[idx] = src;
    }
  }
}

// Compact the occupied orbitals of a spin string into smem (ascending).
__device__ __forceinline__ void occ_list(uint64_t s, int n, int* occ) {
  const int lane = threadIdx.x & 31;
  int base = 0;
  for (int p0 = 0; p0 < n; p0 += 32) {
    int p = p0 + lane;
    bool o = p < n && ((s >> p) & 1ull);
    unsigned m = __ballot_sync(0xffffffffu, o);
    if (o) occ[base + __popc(m & ((1u << lane) - 1u))] = p;
    base += __popc(m);
  }
  __syncwarp();
}

// Largest L with mag[L-1]*absc > eps1 (mag sorted descending).
__device__ __forceinline__ int prefix_len(const double* __restrict__ mag, int len, double absc, double eps1) {
  int lo = 0, hi = len;       // invariant: entries [0,lo) pass, [hi,len) fail
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (mag[mid] * absc > eps1) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Doubles, planning pass: one warp per determinant (dynamic queue).  For
// every occupied pair the length L of the list prefix with |v||c_i| > eps1
// is found by binary search, and the prefix is cut into work items of at
// most WALK_CHUNK entries, so that a determinant with a large coefficient
// (whose prefixes cover most of the lists) is spread over many warps.
__global__ void __launch_bounds__(SEL_WARPS * 32) k_walk_plan(WalkArgs A) {
  // shared: list maxima (n*n + n(n-1)/2 doubles), then the triangular
  // decode table t -> (lo, hi) of occupied-pair indices (bytes)
  extern __shared__ double s_dyn[];
  __shared__ int s_occ[SEL_WARPS][2][HCI_MAXORB];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nmax = A.n * A.n + A.n * (A.n - 1) / 2;
  double* s_max = s_dyn;
  unsigned char* s_tlo = reinterpret_cast<unsigned char*>(s_dyn + nmax);
  const int ntri = HCI_MAXORB * (HCI_MAXORB - 1) / 2;
  unsigned char* s_thi = s_tlo + ntri;
  for (int t = threadIdx.x; t < nmax; t += blockDim.x) s_max[t] = A.list_max[t];
  for (int t = threadIdx.x; t < ntri; t += blockDim.x) {
    int lo, hi;
    tri_decode_dev(t, lo, hi);
    s_tlo[t] = (unsigned char)lo;
    s_thi[t] = (unsigned char)hi;
  }
  __syncthreads();
  int* occA = s_occ[w][0];
  int* occB = s_occ[w][1];
  const int Paa = A.na * (A.na - 1) / 2, Pbb = A.nb * (A.nb - 1) / 2, Pab = A.na * A.nb;
  const int P = Paa + Pbb + Pab;
  const int nn = A.n * A.n;
  while (true) {
    unsigned long long i = 0;
    if (lane == 0) i = atomicAdd(&A.counter[1], 1ull);
    i = __shfl_sync(0xffffffffu, i, 0);
    if ((int64_t)i >= A.nV) break;
    const double absc = fabs(A.c[i]);
    if (!A.accept_all && !(A.max_dbl * absc > A.eps1)) continue;
    const ulonglong2 k = A.keys[i];
    occ_list(k.x, A.n, occA);
    occ_list(k.y, A.n, occB);
    for (int base = 0; base < P; base += 32) {
      int t = base + lane;
      int kind = -1, p = 0, q = 0, L = 0;
      int listid = 0;
      if (t < P) {
        int len;
        double first;
        const double* mag;
        if (t < Paa) {
          p = occA[s_tlo[t]]; q = occA[s_thi[t]]; kind = 0;
          listid = q * (q - 1) / 2 + p;
          first = s_max[nn + listid];
          mag = A.same_mag + (int64_t)listid * A.Ls; len = A.Ls;
        } else if (t < Paa + Pbb) {
          p = occB[s_tlo[t - Paa]]; q = occB[s_thi[t - Paa]]; kind = 1;
          listid = q * (q - 1) / 2 + p;
          first = s_max[nn + listid];
          mag = A.same_mag + (int64_t)listid * A.Ls; len = A.Ls;
        } else {
          int u = t - Paa - Pbb;
          p = occA[u / A.nb]; q = occB[u % A.nb]; kind = 2;
          listid = p * A.n + q;
          first = s_max[listid];
          mag = A.opp_mag + (int64_t)listid * A.Lo; len = A.Lo;
        }
        if (A.accept_all) L = len;
        else if (first * absc > A.eps1) L = prefix_len(mag, len, absc, A.eps1);
      }
      {
        unsigned long long tot = (unsigned long long)L;
        for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        if (lane == 0 && tot) atomicAdd(&A.walkstat[0], tot);
      }
      // work items of at most WALK_CHUNK entries (det, kind|p|q|list, start, end)
      int nit = L > 0 ? (L + WALK_CHUNK - 1) / WALK_CHUNK : 0;
      int incl = nit;
      for (int o = 1; o < 32; o <<= 1) {
        int t2 = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t2;
      }
      const int tot_it = __shfl_sync(0xffffffffu, incl, 31);
      if (tot_it > 0) {
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(A.nitems, (unsigned long long)tot_it);
        base = __shfl_sync(0xffffffffu, base, 31);
        const int code = kind | (p << 2) | (q << 8) | (listid << 14);
        for (int j = 0; j < nit; ++j) {
          const unsigned long long idx = base + (incl - nit) + j;
          if ((int64_t)idx < A.item_cap)
            A.items[idx] = make_int4((int)i, code, j * WALK_CHUNK, min(L, (j + 1) * WALK_CHUNK));
        }
      }
    }
  }
}

// Walk the planned list ranges: one warp per work item; every target whose
// orbitals are empty in the source determinant is emitted.
__global__ void __launch_bounds__(SEL_WARPS * 32) k_walk_exec(WalkArgs A, int64_t nitems) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = warp; it < nitems; it += nwarps) {
    const int4 w = A.items[it];
    const ulonglong2 k = A.keys[w.x];
    const int sk = w.y & 3, sp = (w.y >> 2) & 63, sq = (w.y >> 8) & 63, sl = w.y >> 14;
    const uint16_t* tg = sk == 2 ? A.opp_tgt + (int64_t)sl * A.Lo : A.same_tgt + (int64_t)sl * A.Ls;
    const double ci = A.vals ? A.c[w.x] : 0.0;
    const int64_t n = A.n;
    for (int k0 = w.z; k0 < w.w; k0 += 32) {
      const int e = k0 + lane;
      bool emit = false;
      ulonglong2 key = k;
      double term = 0.0, elem = 0.0;
      if (e < w.w) {
        const uint16_t tt = tg[e];
        const int r = tt & 0xff, s2 = tt >> 8;
        if (sk == 0) {
          if (!((k.x >> r) & 1ull) && !((k.x >> s2) & 1ull)) {
            emit = true;
            key.x = k.x ^ (1ull << sp) ^ (1ull << sq) ^ (1ull << r) ^ (1ull << s2);
          }
        } else if (sk == 1) {
          if (!((k.y >> r) & 1ull) && !((k.y >> s2) & 1ull)) {
            emit = true;
            key.y = k.y ^ (1ull << sp) ^ (1ull << sq) ^ (1ull << r) ^ (1ull << s2);
          }
        } else {
          if (!((k.x >> r) & 1ull) && !((k.y >> s2) & 1ull)) {
            emit = true;
            key.x = k.x ^ (1ull << sp) ^ (1ull << r);
            key.y = k.y ^ (1ull << sq) ^ (1ull << s2);
          }
        }
        if (emit && A.vals) {
          // signed <D_a|H|D_i> (same rule as the graph's elements), times c_i
          double v;
          if (sk == 2) {
            v = exc_phase(k.x, sp, r) * exc_phase(k.y, sq, s2) * A.eri[((sp * n + r) * n + sq) * n + s2];
          } else {
            const uint64_t s0 = sk == 0 ? k.x : k.y;
            const double ph = exc_phase(s0, sp, r) * exc_phase(s0 ^ (1ull << sp) ^ (1ull << r), sq, s2);
            v = ph * (A.eri[((sp * n + r) * n + sq) * n + s2] - A.eri[((sp * n + s2) * n + sq) * n + r]);
          }
          term = v * ci;
          elem = v;
          emit = pt_keep(A, key, term);
        }
      }
      warp_emit(emit, key, A.srcs ? elem : term, w.x, A);
    }
  }
}

// Bound on |H_ai| of the single p->r (spin S) of a determinant D from the
// aufbau reference R: H = F_R + sum over the orbitals where D and R differ of
// +-(pr|kk)-(pk|kr) (same spin) or +-(pr|kk) (other spin), so |H| is at most
// |F_R| plus the absolute values of those few terms; the margin covers the
// rounding of both sums (at most 2n+1 terms bounded by the loose bound B).
__device__ __forceinline__ double single_tight(const WalkArgs& A, int spin, int p, int r, uint64_t s, uint64_t o,
                                               double B) {
  const int n = A.n;
  const uint64_t ds = s ^ (spin == 0 ? A.ref_a : A.ref_b);
  const uint64_t dot = o ^ (spin == 0 ? A.ref_b : A.ref_a);
  const double* js = A.jk_same + ((int64_t)p * n + r) * n;
  const double* jo = A.j_opp + ((int64_t)p * n + r) * n;
  double t = fabs(A.f_ref[((int64_t)spin * n + p) * n + r]);
  uint64_t x = ds;
  while (x) {
    const int k = __ffsll((long long)x) - 1;
    x &= x - 1;
    t += fabs(js[k]);
  }
  x = dot;
  while (x) {
    const int k = __ffsll((long long)x) - 1;
    x &= x - 1;
    t += fabs(jo[k]);
  }
  return (t + 1e-13 * B) * (1.0 + 1e-12);
}

// Singles: one warp per determinant; each lane screens (p->r) with the
// determinant-independent bound, then evaluates H_ai exactly in the same
// summation order as the textbook rule (k ascending, same spin then
// opposite spin per k).
__global__ void __launch_bounds__(SEL_WARPS * 32) k_singles(WalkArgs A) {
  extern __shared__ double s_bound[];          // n*n single-excitation bounds
  __shared__ int s_ov[SEL_WARPS][2][2][HCI_MAXORB];   // [warp][spin][occ/vir][]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = A.n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) s_bound[t] = A.single_bound[t];
  __syncthreads();
  const int Pa = A.na * (n - A.na), Pb = A.nb * (n - A.nb);
  const int P = Pa + Pb;
  while (true) {
    unsigned long long i = 0;
    if (lane == 0) i = atomicAdd(&A.counter[1], 1ull);
    i = __shfl_sync(0xffffffffu, i, 0);
    if ((int64_t)i >= A.nV) break;
    const double absc = fabs(A.c[i]);
    if (!A.accept_all && !(A.max_single * absc > A.eps1)) continue;
    const ulonglong2 k = A.keys[i];
    for (int sp = 0; sp < 2; ++sp) {
      const uint64_t x = sp == 0 ? k.x : k.y;
      int bo = 0, bv = 0;
      for (int p0 = 0; p0 < n; p0 += 32) {
        const int pp = p0 + lane;
        const bool in = pp < n;
        const bool o = in && ((x >> pp) & 1ull);
        const unsigned mo = __ballot_sync(0xffffffffu, o);
        const unsigned mv = __ballot_sync(0xffffffffu, in && !o);
        const unsigned lt = (1u << lane) - 1u;
        if (o) s_ov[w][sp][0][bo + __popc(mo & lt)] = pp;
        if (in && !o) s_ov[w][sp][1][bv + __popc(mv & lt)] = pp;
        bo += __popc(mo);
        bv += __popc(mv);
      }
    }
    __syncwarp();
    for (int base = 0; base < P; base += 32) {
      int t = base + lane;
      bool emit = false, exact = false;
      ulonglong2 key = k;
      double term = 0.0, elem = 0.0;
      if (t < P) {
        int spin = t < Pa ? 0 : 1;
        int u = spin == 0 ? t : t - Pa;
        uint64_t s = spin == 0 ? k.x : k.y;
        uint64_t o = spin == 0 ? k.y : k.x;
        int nocc = spin == 0 ? A.na : A.nb;
        int nvirt = n - nocc;
        const int p = s_ov[w][spin][0][u / nvirt], r = s_ov[w][spin][1][u % nvirt];
        if (A.accept_all && !A.vals) {
          emit = true;
        } else if (A.vals) {
          // perturbative mode: the element from the aufbau value plus the
          // orbitals where the strings differ (no bit-exact decision needed)
          if (A.accept_all || s_bound[p * n + r] * absc > A.eps1) {
            const uint64_t rs = spin == 0 ? A.ref_a : A.ref_b, ro = spin == 0 ? A.ref_b : A.ref_a;
            const double* js = A.jk_same + ((int64_t)p * n + r) * n;
            const double* jo = A.j_opp + ((int64_t)p * n + r) * n;
            double v = A.f_ref[((int64_t)spin * n + p) * n + r];
            for (uint64_t mm = s & ~rs; mm; mm &= mm - 1) v += js[__ffsll((long long)mm) - 1];
            for (uint64_t mm = rs & ~s; mm; mm &= mm - 1) v -= js[__ffsll((long long)mm) - 1];
            for (uint64_t mm = o & ~ro; mm; mm &= mm - 1) v += jo[__ffsll((long long)mm) - 1];
            for (uint64_t mm = ro & ~o; mm; mm &= mm - 1) v -= jo[__ffsll((long long)mm) - 1];
            elem = exc_phase(s, p, r) * v;
            term = elem * A.c[i];
            emit = true;
          }
        } else if (A.accept_all || (s_bound[p * n + r] * absc > A.eps1 &&
                                    single_tight(A, spin, p, r, s, o, s_bound[p * n + r]) * absc > A.eps1)) {
          exact = true;
          double v = A.h[p * n + r];
          const double* js = A.jk_same + ((int64_t)p * n + r) * n;
          const double* jo = A.j_opp + ((int64_t)p * n + r) * n;
          for (int x = 0; x < n; ++x) {
            if ((s >> x) & 1ull) v += js[x];
            if ((o >> x) & 1ull) v += jo[x];
          }
          emit = fabs(v) * absc > A.eps1;
          elem = exc_phase(s, p, r) * v;
          term = elem * A.c[i];
        }
        if (emit) {
          uint64_t ns = s ^ (1ull << p) ^ (1ull << r);
          if (spin == 0) key.x = ns; else key.y = ns;
          if (A.vals) emit = pt_keep(A, key, term);
        }
      }
      // exact evaluations counted once per warp (one atomic, not 32)
      const unsigned mex = __ballot_sync(0xffffffffu, exact);
      if (lane == 0 && mex) atomicAdd(&A.walkstat[1], (unsigned long long)__popc(mex));
      warp_emit(emit, key, A.srcs ? elem : term, (int)i, A);
    }
  }
}

__device__ __forceinline__ bool key_less(ulonglong2 a, ulonglong2 b) {
  return a.x < b.x || (a.x == b.x && a.y < b.y);
}
__device__ __forceinline__ bool key_eq(ulonglong2 a, ulonglong2 b) { return a.x == b.x && a.y == b.y; }

// number of elements of sorted arr[0,n) strictly less than key
__device__ __forceinline__ int64_t lower_bound(const ulonglong2* __restrict__ arr, int64_t n, ulonglong2 key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (key_less(arr[mid], key)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// flag = first of its run in the sorted candidates and not already in V
// c[m + t] = c[t] with the alpha and beta strings exchanged
__global__ void k_flip_append(ulonglong2* __restrict__ c, int64_t m) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    const ulonglong2 k = c[t];
    c[m + t] = make_ulonglong2(k.y, k.x);
  }
}

__global__ void k_flag_new(const ulonglong2* __restrict__ cand, int64_t m, const ulonglong2* __restrict__ V,
                           int64_t nV, int64_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 k = cand[i];
    int64_t f = 0;
    if (i == 0 || !key_eq(k, cand[i - 1])) {
      int64_t pos = lower_bound(V, nV, k);
      f = (pos < nV && key_eq(V[pos], k)) ? 0 : 1;
    }
    flag[i] = f;
  }
}

__global__ void k_compact(const ulonglong2* __restrict__ cand, int64_t m, const int64_t* __restrict__ flag,
                          const int64_t* __restrict__ pos, ulonglong2* __restrict__ out, int64_t cap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (flag[i] && pos[i] < cap) out[pos[i]] = cand[i];
  }
}

__global__ void k_merge_old(const ulonglong2* __restrict__ V, const double* __restrict__ c, int64_t nV,
                            const ulonglong2* __restrict__ N, int64_t nN, ulonglong2* __restrict__ out,
                            double* __restrict__ outc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 k = V[i];
    int64_t pos = i + lower_bound(N, nN, k);
    out[pos] = k;
    if (outc) outc[pos] = c ? c[i] : 0.0;
  }
}

__global__ void k_merge_new(const ulonglong2* __restrict__ V, int64_t nV, const ulonglong2* __restrict__ N,
                            int64_t nN, ulonglong2* __restrict__ out, double* __restrict__ outc) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nN; j += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 k = N[j];
    int64_t pos = j + lower_bound(V, nV, k);
    out[pos] = k;
    if (outc) outc[pos] = 0.0;
  }
}

}  // namespace

static hci_status run_walk(hci_ctx* ctx, WalkArgs& A, int64_t* total) {
  HCI_TRY(ensure_buf(ctx, ctx->s_walkstat, 64));
  A.walkstat = bp<unsigned long long>(ctx->s_walkstat);
  A.nitems = A.walkstat + 2;
  HCI_CUDA(ctx, cudaMemsetAsync(A.walkstat, 0, 16, ctx->st));
  prof_tic(ctx, HCI_PH_WALK);
  HCI_CUDA(ctx, cudaMemsetAsync(A.counter, 0, 16, ctx->st));
  const int grid = ctx->nsm * 8;
  const size_t smw = (size_t)(A.n * A.n + A.n * (A.n - 1) / 2) * 8 + HCI_MAXORB * (HCI_MAXORB - 1);
  HCI_CUDA(ctx, cudaFuncSetAttribute(k_walk_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
  for (int attempt = 0; attempt < 2; ++attempt) {
    HCI_TRY(ensure_buf(ctx, ctx->s_items, (size_t)(ctx->s_items.bytes > 0 ? ctx->s_items.bytes : (1 << 20) * 16)));
    A.items = bp<int4>(ctx->s_items);
    A.item_cap = (int64_t)(ctx->s_items.bytes / 16);
    HCI_CUDA(ctx, cudaMemsetAsync(A.counter + 1, 0, 8, ctx->st));
    HCI_CUDA(ctx, cudaMemsetAsync(A.nitems, 0, 8, ctx->st));
    HCI_LAUNCH(k_walk_plan, grid, SEL_WARPS * 32, smw, ctx->st)(A);
    HCI_CUDA(ctx, cudaGetLastError());
    unsigned long long ni = 0;
    HCI_CUDA(ctx, cudaMemcpyAsync(&ni, A.nitems, 8, cudaMemcpyDeviceToHost, ctx->st));
    HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
    if ((int64_t)ni <= A.item_cap) {
      if (ni > 0) HCI_LAUNCH(k_walk_exec, grid, SEL_WARPS * 32, 0, ctx->st)(A, (int64_t)ni);
      break;
    }
    HCI_TRY(ensure_buf(ctx, ctx->s_items, (size_t)(ni + ni / 8 + 1024) * 16));
  }
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_WALK);
  prof_tic(ctx, HCI_PH_SINGLES);
  HCI_CUDA(ctx, cudaMemsetAsync(A.counter + 1, 0, 8, ctx->st));
  HCI_CUDA(ctx, cudaFuncSetAttribute(k_singles, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
  HCI_LAUNCH(k_singles, grid, SEL_WARPS * 32, (size_t)A.n * A.n * 8, ctx->st)(A);
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_SINGLES);
  unsigned long long cnt = 0, ws[2] = {0, 0};
  HCI_CUDA(ctx, cudaMemcpyAsync(&cnt, A.counter, 8, cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaMemcpyAsync(ws, A.walkstat, 16, cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  ctx->st_counts[HCI_ST_WALK_ENTRIES] += (int64_t)ws[0];
  ctx->st_counts[HCI_ST_SINGLES_EXACT] += (int64_t)ws[1];
  *total = (int64_t)cnt;
  return HCI_OK;
}

extern "C" hci_status hci_select(hci_ctx* ctx, double eps1, const uint64_t* keys, const double* c, int64_t nV,
                                 uint64_t* new_keys, int64_t cap, int64_t* n_new) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_select: null context");
  if (!n_new) return hci_fail(ctx, HCI_ERR_INVALID, "hci_select: n_new is NULL");
  *n_new = 0;
  if (nV < 0 || cap < 0) return hci_fail(ctx, HCI_ERR_INVALID, "hci_select: negative size");
  if (nV > 0 && (!keys || !c)) return hci_fail(ctx, HCI_ERR_INVALID, "hci_select: null keys or c");
  if (cap > 0 && !new_keys) return hci_fail(ctx, HCI_ERR_INVALID, "hci_select: null new_keys");
  if (nV == 0) return HCI_OK;
  HCI_TRY(hci_build_lists(ctx));
  int ok = 0;
  HCI_TRY(check_sorted(ctx, keys, nV, &ok));
  if (!ok) return hci_fail(ctx, HCI_ERR_INVALID, "hci_select: keys are not strictly ascending");
  Lists& L = ctx->lists;
  WalkArgs A;
  A.n = ctx->n; A.na = ctx->na; A.nb = ctx->nb;
  A.keys = reinterpret_cast<const ulonglong2*>(keys);
  A.c = c; A.nV = nV; A.eps1 = eps1; A.accept_all = eps1 <= 0.0 ? 1 : 0;
  A.opp_mag = bp<double>(L.opp_mag); A.opp_tgt = bp<uint16_t>(L.opp_tgt); A.Lo = L.len_opp;
  A.same_mag = bp<double>(L.same_mag); A.same_tgt = bp<uint16_t>(L.same_tgt); A.Ls = L.len_same;
  A.max_dbl = L.max_opp > L.max_same ? L.max_opp : L.max_same;
  A.h = bp<double>(ctx->h); A.jk_same = bp<double>(ctx->jk_same); A.j_opp = bp<double>(ctx->j_opp);
  A.single_bound = bp<double>(L.single_bound); A.max_single = L.max_single;
  A.list_max = bp<double>(L.list_max);
  A.f_ref = bp<double>(L.f_ref);
  A.ref_a = ctx->na == 64 ? ~0ull : ((1ull << ctx->na) - 1ull);
  A.ref_b = ctx->nb == 64 ? ~0ull : ((1ull << ctx->nb) - 1ull);
  A.vals = nullptr; A.srcs = nullptr; A.npart = 1; A.part = 0; A.eri = bp<double>(ctx->eri);
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  A.counter = bp<unsigned long long>(ctx->s_counter);
  // candidate buffer: grow and rerun when the first guess overflows
  int64_t guess = ctx->s_cand.bytes / 16;
  if (guess < (int64_t)1 << 16) guess = (int64_t)1 << 16;
  HCI_TRY(ensure_buf(ctx, ctx->s_cand, (size_t)guess * 16));
  A.out = bp<ulonglong2>(ctx->s_cand);
  A.cap = (int64_t)(ctx->s_cand.bytes / 16);
  int64_t m = 0;
  HCI_TRY(run_walk(ctx, A, &m));
  if (m > A.cap) {
    HCI_TRY(ensure_buf(ctx, ctx->s_cand, (size_t)(m + m / 8 + 1024) * 16));
    A.out = bp<ulonglong2>(ctx->s_cand);
    A.cap = (int64_t)(ctx->s_cand.bytes / 16);
    int64_t m2 = 0;
    HCI_TRY(run_walk(ctx, A, &m2));
    if (m2 != m) return hci_fail(ctx, HCI_ERR_CUDA, "hci_select: candidate count changed between runs");
  }
  if (ctx->spin_parity != 0 && m > 0) {
    // spin parity: every selected determinant brings its spin-flip partner
    HCI_TRY(ensure_buf(ctx, ctx->s_cand2, (size_t)2 * m * 16));
    HCI_CUDA(ctx, cudaMemcpyAsync(ctx->s_cand2.p, ctx->s_cand.p, (size_t)m * 16, cudaMemcpyDeviceToDevice, ctx->st));
    HCI_LAUNCH(k_flip_append, grid_for(m, 256), 256, 0, ctx->st)(bp<ulonglong2>(ctx->s_cand2), m);
    HCI_CUDA(ctx, cudaGetLastError());
    std::swap(ctx->s_cand, ctx->s_cand2);
    m *= 2;
  }
  ctx->last_candidates = m;
  ctx->st_counts[HCI_ST_SELECT_CALLS] += 1;
  ctx->st_counts[HCI_ST_SELECT_SOURCES] += nV;
  ctx->st_counts[HCI_ST_CANDIDATES] += m;
  if (m == 0) return HCI_OK;
  prof_tic(ctx, HCI_PH_DEDUP);
  HCI_TRY(ensure_buf(ctx, ctx->s_cand2, (size_t)m * 16));
  HCI_TRY(sort_keys(ctx, bp<uint64_t>(ctx->s_cand), bp<uint64_t>(ctx->s_cand2), m, ctx->n, ctx->n));
  HCI_TRY(ensure_buf(ctx, ctx->s_flags, (size_t)(2 * m + 1) * 8));
  int64_t* flag = bp<int64_t>(ctx->s_flags);
  int64_t* pos = flag + m;
  int64_t* total = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 16);
  HCI_LAUNCH(k_flag_new, grid_for(m, 256), 256, 0, ctx->st)(bp<ulonglong2>(ctx->s_cand), m,
                                                    reinterpret_cast<const ulonglong2*>(keys), nV, flag);
  HCI_CUDA(ctx, cudaGetLastError());
  HCI_TRY(scan_i64(ctx, flag, pos, m, total));
  prof_toc(ctx, HCI_PH_DEDUP);
  int64_t cnt = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&cnt, total, 8, cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  *n_new = cnt;
  if (cnt > cap)
    return hci_fail(ctx, HCI_ERR_CAPACITY, "hci_select: %lld new determinants exceed cap %lld", (long long)cnt,
                    (long long)cap);
  HCI_LAUNCH(k_compact, grid_for(m, 256), 256, 0, ctx->st)(bp<ulonglong2>(ctx->s_cand), m, flag, pos,
                                                   reinterpret_cast<ulonglong2*>(new_keys), cap);
  HCI_CUDA(ctx, cudaGetLastError());
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  return HCI_OK;
}

extern "C" hci_status hci_merge(hci_ctx* ctx, const uint64_t* keys, const double* c, int64_t nV,
                                const uint64_t* new_keys, int64_t n_new, uint64_t* out_keys, double* out_c) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_merge: null context");
  if (nV < 0 || n_new < 0) return hci_fail(ctx, HCI_ERR_INVALID, "hci_merge: negative size");
  if ((nV + n_new) > 0 && !out_keys) return hci_fail(ctx, HCI_ERR_INVALID, "hci_merge: null out_keys");
  const ulonglong2* V = reinterpret_cast<const ulonglong2*>(keys);
  const ulonglong2* N = reinterpret_cast<const ulonglong2*>(new_keys);
  ulonglong2* O = reinterpret_cast<ulonglong2*>(out_keys);
  prof_tic(ctx, HCI_PH_MERGE);
  if (nV > 0)
    HCI_LAUNCH(k_merge_old, grid_for(nV, 256), 256, 0, ctx->st)(V, c, nV, N, n_new, O, out_c);
  if (n_new > 0)
    HCI_LAUNCH(k_merge_new, grid_for(n_new, 256), 256, 0, ctx->st)(V, nV, N, n_new, O, out_c);
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_MERGE);
  return HCI_OK;
}

// ---------------------------------------------------------------------------
// Second-order Epstein-Nesbet correction with screening (Sec. II.B,
// Eq. pt_hci): the walk and the singles emit every target D_a with its term
// H_ai c_i when |H_ai c_i| > eps2; the (target, term) pairs are sorted by
// target, targets in V are dropped, and each remaining target contributes
// (sum of its terms)^2 / (E0 - H_aa).  The targets are processed in hash
// classes so that at most max_pairs pairs are held at once.
// ---------------------------------------------------------------------------
namespace {

// Aufbau reference R for diagonal elements by differences, over spin
// orbitals k (alpha 0..n-1, beta n..2n-1): g_kl = (kk|ll) - [same spin] (kl|lk),
// F_k = h_kk + sum_{l in R, l != k} g_kl, E_R = e_core + sum_{k in R} h_kk +
// sum_{k<l in R} g_kl.  out = [E_R, F (2n), g (2n x 2n)].
__global__ void k_pt2_ref(int n, const double* __restrict__ h, const double* __restrict__ eri, double ecore,
                          uint64_t ra, uint64_t rb, double* __restrict__ out) {
  const int m = 2 * n;
  double* F = out + 1;
  double* g = out + 1 + m;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int k = t / m, l = t % m, p = k % n, q = l % n;
    double v = eri[(((int64_t)p * n + p) * n + q) * n + q];
    if ((k < n) == (l < n)) v -= eri[(((int64_t)p * n + q) * n + q) * n + p];
    g[t] = k == l ? 0.0 : v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    double f = h[(k % n) * n + (k % n)];
    for (int l = 0; l < m; ++l) {
      const bool occ = l < n ? ((ra >> l) & 1ull) : ((rb >> (l - n)) & 1ull);
      if (occ && l != k) f += g[k * m + l];
    }
    F[k] = f;
  }
  if (threadIdx.x == 0) {
    double e = ecore;
    for (int k = 0; k < m; ++k) {
      if (!(k < n ? ((ra >> k) & 1ull) : ((rb >> (k - n)) & 1ull))) continue;
      e += h[(k % n) * n + (k % n)];
      for (int l = k + 1; l < m; ++l)
        if (l < n ? ((ra >> l) & 1ull) : ((rb >> (l - n)) & 1ull)) e += g[k * m + l];
    }
    out[0] = e;
  }
}

// H_aa = E_R + sum_k d_k F_k + sum_{k<l} d_k d_l g_kl over the spin orbitals
// where D_a differs from R (d = +1 occupied in D_a only, -1 in R only)
__device__ __forceinline__ double pt2_diag(const double* s_ref, int n, ulonglong2 key, uint64_t ra, uint64_t rb) {
  const int m = 2 * n;
  const double* F = s_ref + 1;
  const double* g = s_ref + 1 + m;
  const uint64_t da = key.x ^ ra, db = key.y ^ rb;
  double e = s_ref[0];
  for (uint64_t x = da; x; x &= x - 1) {
    const int k = __ffsll((long long)x) - 1;
    const double dk = ((key.x >> k) & 1ull) ? 1.0 : -1.0;
    e += dk * F[k];
    for (uint64_t y = x & (x - 1); y; y &= y - 1) {
      const int l = __ffsll((long long)y) - 1;
      e += dk * (((key.x >> l) & 1ull) ? 1.0 : -1.0) * g[k * m + l];
    }
    for (uint64_t y = db; y; y &= y - 1) {
      const int l = __ffsll((long long)y) - 1;
      e += dk * (((key.y >> l) & 1ull) ? 1.0 : -1.0) * g[k * m + n + l];
    }
  }
  for (uint64_t x = db; x; x &= x - 1) {
    const int k = __ffsll((long long)x) - 1;
    const double dk = ((key.y >> k) & 1ull) ? 1.0 : -1.0;
    e += dk * F[n + k];
    for (uint64_t y = x & (x - 1); y; y &= y - 1) {
      const int l = __ffsll((long long)y) - 1;
      e += dk * (((key.y >> l) & 1ull) ? 1.0 : -1.0) * g[(n + k) * m + n + l];
    }
  }
  return e;
}

// On the first pair of every run of equal targets (sorted): the run's terms
// summed, the target dropped when it is in V, else contrib = sum^2 /
// (e0 - H_aa) and ext = 1; zero on every other pair.
__global__ void k_pt2_terms(const ulonglong2* __restrict__ t, const double* __restrict__ v, int64_t m,
                            const ulonglong2* __restrict__ V, int64_t nV, int n, const double* __restrict__ ref,
                            uint64_t ra, uint64_t rb, double e0, double* __restrict__ contrib,
                            int64_t* __restrict__ ext, double* __restrict__ dpair, const double* __restrict__ cvec,
                            const int32_t* __restrict__ src) {
  extern __shared__ double s_ref[];
  const int nref = 1 + 2 * n + 4 * n * n;
  for (int u = threadIdx.x; u < nref; u += blockDim.x) s_ref[u] = ref[u];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double cv = 0.0;
    int64_t e = 0;
    const ulonglong2 key = t[i];
    if (i == 0 || !key_eq(key, t[i - 1])) {
      const int64_t pos = lower_bound(V, nV, key);
      double da = 0.0;
      int64_t end = i + 1;
      if (!(pos < nV && key_eq(V[pos], key))) {
        double num = 0.0;
        for (end = i; end < m && key_eq(t[end], key); ++end) num += src ? v[end] * cvec[src[end]] : v[end];
        da = num / (e0 - pt2_diag(s_ref, n, key, ra, rb));
        cv = num * da;
        e = 1;
      } else if (dpair) {
        while (end < m && key_eq(t[end], key)) ++end;
      }
      // first-order coefficient d_a on every pair of the run (0 for D_a in V)
      if (dpair)
        for (int64_t j = i; j < end; ++j) dpair[j] = da;
    }
    contrib[i] = cv;
    ext[i] = e;
  }
}

// dE2/dc_i = 2 sum over the screened pairs of d_a H_ai (the pairs fixed)
__global__ void k_pt2_grad(const int32_t* __restrict__ src, const double* __restrict__ elem,
                           const double* __restrict__ d, int64_t m, double* __restrict__ g) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
    if (d[j] != 0.0) atomicAdd(&g[src[j]], 2.0 * d[j] * elem[j]);
}

constexpr int PT2_SUM_BLOCKS = 1024;

// part[b] = sum of a[] over block b's contiguous slice, in order
__global__ void k_sum_slices_d(const double* __restrict__ a, int64_t m, double* __restrict__ part) {
  __shared__ double red[256];
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < m ? lo + per : m;
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += a[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_parts_d(const double* __restrict__ part, int np, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < np; ++b) s += part[b];
    *out = s;
  }
}

}  // namespace

// Walk arguments of the perturbative modes: sources keys/c (nV of them),
// terms kept when |H_ai c_i| > eps (every single and double when eps < 0).
static hci_status pt_walk_args(hci_ctx* ctx, WalkArgs& A, const uint64_t* keys, const double* c, int64_t nV,
                               double eps) {
  Lists& L = ctx->lists;
  A = WalkArgs{};
  A.n = ctx->n; A.na = ctx->na; A.nb = ctx->nb;
  A.keys = reinterpret_cast<const ulonglong2*>(keys);
  A.c = c; A.nV = nV; A.eps1 = eps; A.accept_all = eps <= 0.0 ? 1 : 0;
  A.opp_mag = bp<double>(L.opp_mag); A.opp_tgt = bp<uint16_t>(L.opp_tgt); A.Lo = L.len_opp;
  A.same_mag = bp<double>(L.same_mag); A.same_tgt = bp<uint16_t>(L.same_tgt); A.Ls = L.len_same;
  A.max_dbl = L.max_opp > L.max_same ? L.max_opp : L.max_same;
  A.h = bp<double>(ctx->h); A.jk_same = bp<double>(ctx->jk_same); A.j_opp = bp<double>(ctx->j_opp);
  A.single_bound = bp<double>(L.single_bound); A.max_single = L.max_single;
  A.list_max = bp<double>(L.list_max);
  A.f_ref = bp<double>(L.f_ref);
  A.ref_a = ctx->na == 64 ? ~0ull : ((1ull << ctx->na) - 1ull);
  A.ref_b = ctx->nb == 64 ? ~0ull : ((1ull << ctx->nb) - 1ull);
  A.eri = bp<double>(ctx->eri);
  A.srcs = nullptr;
  A.vals = nullptr;
  A.npart = 1;
  A.part = 0;
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  A.counter = bp<unsigned long long>(ctx->s_counter);
  return HCI_OK;
}

extern "C" hci_status hci_pt2(hci_ctx* ctx, double eps2, const uint64_t* keys, const double* c, int64_t nV,
                              double e0, int64_t max_pairs, double* e2, int64_t* n_ext, double* rdm1_dd,
                              double* rdm2_dd, double* rdm1_dc, double* rdm2_dc, double* grad_c) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_pt2: null context");
  if (!e2) return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2: e2 is NULL");
  *e2 = 0.0;
  if (n_ext) *n_ext = 0;
  if (nV < 0 || max_pairs < 0) return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2: negative size");
  if (nV > 0 && (!keys || !c)) return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2: null keys or c");
  const int nrdm = (rdm1_dd != nullptr) + (rdm2_dd != nullptr) + (rdm1_dc != nullptr) + (rdm2_dc != nullptr);
  if (nrdm != 0 && nrdm != 4) return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2: give all four density matrices or none");
  const bool want_rdm = nrdm == 4;
  const bool want_src = want_rdm || grad_c != nullptr;
  if (grad_c && nV > 0) HCI_CUDA(ctx, cudaMemsetAsync(grad_c, 0, (size_t)nV * 8, ctx->st));
  if (want_rdm) {
    const size_t n2 = (size_t)ctx->n * ctx->n;
    HCI_CUDA(ctx, cudaMemsetAsync(rdm1_dd, 0, n2 * 8, ctx->st));
    HCI_CUDA(ctx, cudaMemsetAsync(rdm2_dd, 0, n2 * n2 * 8, ctx->st));
    HCI_CUDA(ctx, cudaMemsetAsync(rdm1_dc, 0, n2 * 8, ctx->st));
    HCI_CUDA(ctx, cudaMemsetAsync(rdm2_dc, 0, n2 * n2 * 8, ctx->st));
    HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  }
  if (nV == 0) return HCI_OK;
  HCI_TRY(hci_build_lists(ctx));
  int ok = 0;
  HCI_TRY(check_sorted(ctx, keys, nV, &ok));
  if (!ok) return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2: keys are not strictly ascending");
  cudaStream_t st = ctx->st;
  const int n = ctx->n;
  WalkArgs A;
  HCI_TRY(pt_walk_args(ctx, A, keys, c, nV, eps2));
  if (want_rdm) HCI_TRY(pt2_rdm_begin(ctx));
  // aufbau reference of the diagonal elements
  const size_t nref = 1 + 2 * (size_t)n + 4 * (size_t)n * n;
  HCI_TRY(ensure_buf(ctx, ctx->p2_ref, nref * 8 + (PT2_SUM_BLOCKS + 2) * 8));
  double* ref = bp<double>(ctx->p2_ref);
  double* part = ref + nref;
  double* dsum = part + PT2_SUM_BLOCKS;
  HCI_LAUNCH(k_pt2_ref, 1, 256, 0, st)(n, bp<double>(ctx->h), bp<double>(ctx->eri), ctx->ecore, A.ref_a, A.ref_b,
                                       ref);
  HCI_CUDA(ctx, cudaGetLastError());
  const int64_t per = max_pairs > 0 ? max_pairs : ((int64_t)1 << 28);
  double acc = 0.0;
  int64_t next_total = 0;
  // one hash class of targets: walk into the pair buffer (walked again with
  // a larger buffer if it was too small), sort, reduce
  auto run_class = [&](int npart, int pc, int64_t* m_out, bool reduce) -> hci_status {
    A.npart = npart;
    A.part = pc;
    int64_t m = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
      A.out = bp<ulonglong2>(ctx->s_cand);
      A.vals = bp<double>(ctx->p2_vals);
      A.cap = (int64_t)std::min(ctx->s_cand.bytes / 16, ctx->p2_vals.bytes / 8);
      if (want_src) {
        HCI_TRY(ensure_buf(ctx, ctx->p2_src, (size_t)A.cap * 4));
        A.srcs = bp<int32_t>(ctx->p2_src);
      }
      HCI_TRY(run_walk(ctx, A, &m));
      if (m <= A.cap || (npart == 1 && m > per)) break;
      HCI_TRY(ensure_buf(ctx, ctx->s_cand, (size_t)(m + m / 8 + 4096) * 16));
      HCI_TRY(ensure_buf(ctx, ctx->p2_vals, (size_t)(m + m / 8 + 4096) * 8));
    }
    *m_out = m;
    if (npart == 1 && m > per) return HCI_OK;   // too many for one class: the caller splits the targets
    if (m > A.cap) return hci_fail(ctx, HCI_ERR_CUDA, "hci_pt2: pair count changed between walks");
    if (!reduce || m == 0) return HCI_OK;
    HCI_TRY(ensure_buf(ctx, ctx->s_cand2, (size_t)m * 16));
    HCI_TRY(ensure_buf(ctx, ctx->p2_vals2, (size_t)m * 8));
    int32_t* src = nullptr;
    int32_t* src2 = nullptr;
    double* dpair = nullptr;
    if (want_src) {
      HCI_TRY(ensure_buf(ctx, ctx->p2_src2, (size_t)m * 4));
      HCI_TRY(ensure_buf(ctx, ctx->p2_d, (size_t)m * 8));
      src = bp<int32_t>(ctx->p2_src);
      src2 = bp<int32_t>(ctx->p2_src2);
      dpair = bp<double>(ctx->p2_d);
    }
    HCI_TRY(sort_pairs(ctx, bp<uint64_t>(ctx->s_cand), bp<uint64_t>(ctx->s_cand2), bp<double>(ctx->p2_vals),
                       bp<double>(ctx->p2_vals2), src, src2, m, n, n));
    HCI_TRY(ensure_buf(ctx, ctx->s_flags, (size_t)(2 * m + 1) * 8));
    int64_t* ext = bp<int64_t>(ctx->s_flags);
    int64_t* ext_scan = ext + m;
    double* contrib = bp<double>(ctx->p2_vals2);
    const size_t sm = nref * 8;
    HCI_CUDA(ctx, cudaFuncSetAttribute(k_pt2_terms, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HCI_LAUNCH(k_pt2_terms, grid_for(m, 256), 256, sm, st)(bp<ulonglong2>(ctx->s_cand), bp<double>(ctx->p2_vals), m,
                                                          A.keys, nV, n, ref, A.ref_a, A.ref_b, e0, contrib, ext,
                                                          dpair, c, src);
    if (grad_c)
      HCI_LAUNCH(k_pt2_grad, grid_for(m, 256), 256, 0, st)(src, bp<double>(ctx->p2_vals), dpair, m, grad_c);
    if (want_rdm) HCI_TRY(pt2_rdm_pairs(ctx, A.keys, c, bp<ulonglong2>(ctx->s_cand), src, dpair, m));
    HCI_CUDA(ctx, cudaGetLastError());
    HCI_LAUNCH(k_sum_slices_d, PT2_SUM_BLOCKS, 256, 0, st)(contrib, m, part);
    HCI_LAUNCH(k_sum_parts_d, 1, 32, 0, st)(part, PT2_SUM_BLOCKS, dsum);
    int64_t* cnt_dev = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 40);
    HCI_TRY(scan_i64(ctx, ext, ext_scan, m, cnt_dev));
    HCI_CUDA(ctx, cudaGetLastError());
    double hs = 0.0;
    int64_t hc = 0;
    HCI_CUDA(ctx, cudaMemcpyAsync(&hs, dsum, 8, cudaMemcpyDeviceToHost, st));
    HCI_CUDA(ctx, cudaMemcpyAsync(&hc, cnt_dev, 8, cudaMemcpyDeviceToHost, st));
    HCI_CUDA(ctx, cudaStreamSynchronize(st));
    acc += hs;
    next_total += hc;
    return HCI_OK;
  };
  HCI_TRY(ensure_buf(ctx, ctx->s_cand, (size_t)4096 * 16));
  HCI_TRY(ensure_buf(ctx, ctx->p2_vals, (size_t)4096 * 8));
  // all targets at once when they fit max_pairs; else hash classes
  int64_t total = 0;
  HCI_TRY(run_class(1, 0, &total, true));
  if (total > per) {
    const int64_t np64 = (total + per - 1) / per;
    if (np64 > (1 << 20))
      return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2: max_pairs too small for %lld pairs", (long long)total);
    const int npart = (int)np64;
    const int64_t cap = total / npart + total / (8 * (int64_t)npart) + 4096;
    HCI_TRY(ensure_buf(ctx, ctx->s_cand, (size_t)cap * 16));
    HCI_TRY(ensure_buf(ctx, ctx->p2_vals, (size_t)cap * 8));
    for (int pc = 0; pc < npart; ++pc) {
      int64_t m = 0;
      HCI_TRY(run_class(npart, pc, &m, true));
    }
  }
  if (want_rdm) {
    HCI_TRY(pt2_rdm_finish(ctx, rdm1_dd, rdm2_dd, rdm1_dc, rdm2_dc));
    HCI_CUDA(ctx, cudaStreamSynchronize(st));
  }
  *e2 = acc;
  if (n_ext) *n_ext = next_total;
  return HCI_OK;
}

// ---------------------------------------------------------------------------
// Semistochastic second-order correction (Sec. II.B, Eq. semistoc):
// E2 ~ E2^D(eps2_det) + mean over samples of [E2^S(eps2) - E2^S(eps2_det)],
// both stochastic terms of a sample taken from the same draws.  A sample is
// n_draws determinants of V drawn with replacement, D_i with probability
// p_i = W_i / sum W (integer weights W_i proportional to |c_i|); the drawn
// determinants are walked like V in the deterministic correction, and every
// target outside V contributes the unbiased multinomial estimate of the
// cited semistochastic HCI work, grouped as
//   (S^2 - T + (N_d - 1) U) / (N_d (N_d - 1) (E0 - H_aa)),
// S = sum_j f_j x_j, T = sum_j (f_j x_j)^2, U = sum_j f_j x_j^2,
// x_j = H_aj c_j, f_j = w_j / p_j (w_j = times D_j was drawn).
// Draw k of sample s uses the first word r of Philox4x64-10 at counter
// (k, s, 0, 0) and key (seed, 0): u = floor(r sum W / 2^64), and the drawn
// index is the i with prefix_{i-1} <= u < prefix_i of the inclusive prefix
// sums of W.  Weights, prefix sums and the draw are exact integer
// arithmetic, so the draws do not depend on the summation order.
// ---------------------------------------------------------------------------
namespace {

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 64x64->128 multiplications by fixed odd constants, the halves mixed with
// the other two words and the key; the key is bumped by two Weyl
// constants between rounds.
__device__ __forceinline__ uint64_t philox4x64_first(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                     uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B97F4A7C15ull;
      k1 += 0xBB67AE8584CAA73Bull;
    }
    const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
    const uint64_t hi0 = __umul64hi(m0, c0), lo0 = m0 * c0;
    const uint64_t hi1 = __umul64hi(m1, c2), lo1 = m1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return c0;
}

// largest |c_i| (bit pattern of a non-negative double orders like the value)
__global__ void k_abs_max(const double* __restrict__ c, int64_t n, unsigned long long* __restrict__ mx) {
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(c[i]));
    m = b > m ? b : m;
  }
  for (int o = 16; o; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

// W_i = ceil(|c_i| 2^(B - E)), 2^(E-1) <= max|c| < 2^E: W_i >= 1 iff c_i != 0, W_i <= 2^B, sum W <= 2^62
__global__ void k_ss_weights(const double* __restrict__ c, int64_t n, const unsigned long long* __restrict__ mx,
                             int B, int64_t* __restrict__ W) {
  int e = 0;
  frexp(__longlong_as_double((long long)*mx), &e);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    W[i] = (int64_t)ceil(ldexp(fabs(c[i]), B - e));
}

// draws: key (x = sample, y = drawn index) for the sort, and the index alone
__global__ void k_ss_draw(const int64_t* __restrict__ excl, int64_t nV,
                          const int64_t* __restrict__ total, uint64_t seed, int64_t nd, int64_t m,
                          ulonglong2* __restrict__ out, int32_t* __restrict__ draws) {
  const uint64_t tot = (uint64_t)*total;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / nd, k = t - s * nd;
    const uint64_t r = philox4x64_first((uint64_t)k, (uint64_t)s, 0ull, 0ull, seed, 0ull);
    const uint64_t u = __umul64hi(r, tot);
    // the i with excl[i] <= u < excl[i] + W[i] is the last i with
    // excl[i] <= u (a zero weight shares its start with the next entry, and
    // the last entry ends at the total > u, so that i has W[i] > 0)
    int64_t lo = 0, hi = nV;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((uint64_t)excl[mid] <= u) lo = mid + 1;
      else hi = mid;
    }
    const int64_t i = lo - 1;
    out[t] = make_ulonglong2((unsigned long long)s, (unsigned long long)i);
    if (draws) draws[t] = (int32_t)i;
  }
}

__global__ void k_run_first(const ulonglong2* __restrict__ k, int64_t m, int64_t* __restrict__ flag) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
    flag[t] = (t == 0 || !key_eq(k[t], k[t - 1])) ? 1 : 0;
}

// distinct (sample, index) runs of the sorted draws: index, sample, first position
__global__ void k_ss_compact(const ulonglong2* __restrict__ k, int64_t m, const int64_t* __restrict__ flag,
                             const int64_t* __restrict__ pos, int32_t* __restrict__ d_idx, int32_t* __restrict__ d_s,
                             int64_t* __restrict__ d_start) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
    if (flag[t]) {
      const int64_t j = pos[t];
      d_idx[j] = (int32_t)k[t].y;
      d_s[j] = (int32_t)k[t].x;
      d_start[j] = t;
    }
}

// seg[s] = first distinct run of sample s (s = 0..ns)
__global__ void k_ss_seg(const int32_t* __restrict__ d_s, int64_t nd, int ns, int64_t* __restrict__ seg) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= ns; s += gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = nd;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (d_s[mid] < s) lo = mid + 1;
      else hi = mid;
    }
    seg[s] = lo;
  }
}

// the sources of one sample: key, c, f = w / p with p = W_i / sum W
__global__ void k_ss_gather(int64_t j0, int64_t j1, int64_t ndist, int64_t m, const int32_t* __restrict__ d_idx,
                            const int64_t* __restrict__ d_start, const ulonglong2* __restrict__ keys,
                            const double* __restrict__ c, const int64_t* __restrict__ W,
                            const int64_t* __restrict__ total, ulonglong2* __restrict__ sk, double* __restrict__ sc,
                            double* __restrict__ sf) {
  const double tot = (double)*total;
  for (int64_t j = j0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < j1;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = (j + 1 < ndist ? d_start[j + 1] : m) - d_start[j];
    const int32_t i = d_idx[j];
    const double p = (double)W[i] / tot;
    sk[j - j0] = keys[i];
    sc[j - j0] = c[i];
    sf[j - j0] = (double)w / p;
  }
}

// On the first pair of every run of equal targets (sorted; element H_aj and
// source j on each pair): targets in V give 0, the others their estimate
// with the eps2 screen (every emitted pair) and with eps2_det.
__global__ void k_ss_terms(const ulonglong2* __restrict__ t, const double* __restrict__ v,
                           const int32_t* __restrict__ src, int64_t m, const ulonglong2* __restrict__ V, int64_t nV,
                           const double* __restrict__ sc, const double* __restrict__ sf, double eps2_det,
                           double nd, int n, const double* __restrict__ ref, uint64_t ra, uint64_t rb, double e0,
                           double* __restrict__ out_t, double* __restrict__ out_d) {
  extern __shared__ double s_ref[];
  const int nref = 1 + 2 * n + 4 * n * n;
  for (int u = threadIdx.x; u < nref; u += blockDim.x) s_ref[u] = ref[u];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double et = 0.0, ed = 0.0;
    const ulonglong2 key = t[i];
    if (i == 0 || !key_eq(key, t[i - 1])) {
      const int64_t pos = lower_bound(V, nV, key);
      if (!(pos < nV && key_eq(V[pos], key))) {
        double S[2] = {0.0, 0.0}, T[2] = {0.0, 0.0}, U[2] = {0.0, 0.0};
        for (int64_t e = i; e < m && key_eq(t[e], key); ++e) {
          const int32_t j = src[e];
          const double x = v[e] * sc[j], f = sf[j];
          for (int k = 0; k < 2; ++k) {
            if (k == 1 && !(fabs(x) > eps2_det)) break;
            S[k] += f * x;
            T[k] += (f * x) * (f * x);
            U[k] += f * x * x;
          }
        }
        const double den = nd * (nd - 1.0) * (e0 - pt2_diag(s_ref, n, key, ra, rb));
        et = (S[0] * S[0] - T[0] + (nd - 1.0) * U[0]) / den;
        ed = (S[1] * S[1] - T[1] + (nd - 1.0) * U[1]) / den;
      }
    }
    out_t[i] = et;
    out_d[i] = ed;
  }
}

}  // namespace

extern "C" hci_status hci_pt2_stochastic(hci_ctx* ctx, const uint64_t* keys, const double* c, int64_t nV, double e0,
                                         double eps2, double eps2_det, int64_t n_draws, int n_samples,
                                         uint64_t seed, int64_t max_pairs, double* result, double* sample_e2,
                                         int32_t* draws) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_pt2_stochastic: null context");
  if (!result) return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2_stochastic: result is NULL");
  result[0] = result[1] = result[2] = 0.0;
  if (nV < 0 || max_pairs < 0) return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2_stochastic: negative size");
  if (n_draws < 2 || n_samples < 1)
    return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2_stochastic: need n_draws >= 2 and n_samples >= 1");
  if (n_draws * (int64_t)n_samples > INT32_MAX)
    return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2_stochastic: n_draws * n_samples exceeds 2^31 - 1");
  if (!(eps2 <= eps2_det)) return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2_stochastic: eps2 must not exceed eps2_det");
  if (nV > INT32_MAX) return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2_stochastic: more than 2^31 - 1 determinants");
  if (sample_e2)
    for (int s = 0; s < 2 * n_samples; ++s) sample_e2[s] = 0.0;
  if (nV == 0) return HCI_OK;
  if (!keys || !c) return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2_stochastic: null keys or c");
  // deterministic part (also checks the keys and builds the lists)
  double e2d = 0.0;
  HCI_TRY(hci_pt2(ctx, eps2_det, keys, c, nV, e0, max_pairs, &e2d, nullptr, nullptr, nullptr, nullptr, nullptr,
                  nullptr));
  cudaStream_t st = ctx->st;
  const int n = ctx->n;
  const int64_t nd = n_draws, m = nd * n_samples;
  // weights, their exclusive prefix sums and total
  HCI_TRY(ensure_buf(ctx, ctx->ss_w, (size_t)(2 * nV + 2) * 8));
  int64_t* W = bp<int64_t>(ctx->ss_w);
  int64_t* excl = W + nV;
  int64_t* total = excl + nV;
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(total + 1);
  HCI_CUDA(ctx, cudaMemsetAsync(mx, 0, 8, st));
  HCI_LAUNCH(k_abs_max, grid_for(nV, 256, ctx->nsm * 8), 256, 0, st)(c, nV, mx);
  // weight scale 2^B: 2^40, or less so that nV 2^B <= 2^62
  int lg = 0;
  while (((int64_t)1 << lg) < nV) ++lg;
  const int B = lg <= 22 ? 40 : 62 - lg;
  HCI_LAUNCH(k_ss_weights, grid_for(nV, 256, ctx->nsm * 8), 256, 0, st)(c, nV, mx, B, W);
  HCI_TRY(scan_i64(ctx, W, excl, nV, total));
  int64_t tot_h = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&tot_h, total, 8, cudaMemcpyDeviceToHost, st));
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  if (tot_h == 0) {   // c = 0: every estimate is 0
    result[2] = e2d;
    result[0] = e2d;
    if (draws) HCI_CUDA(ctx, cudaMemsetAsync(draws, 0, (size_t)m * 4, st));
    return HCI_OK;
  }
  // draws, sorted by (sample, index), and their distinct runs
  HCI_TRY(ensure_buf(ctx, ctx->ss_draw, (size_t)m * 16));
  HCI_TRY(ensure_buf(ctx, ctx->ss_draw2, (size_t)m * 16));
  ulonglong2* dk = bp<ulonglong2>(ctx->ss_draw);
  HCI_LAUNCH(k_ss_draw, grid_for(m, 256, ctx->nsm * 8), 256, 0, st)(excl, nV, total, seed, nd, m, dk, draws);
  int sbits = 1, ibits = 1;
  while (sbits < 32 && ((int64_t)1 << sbits) < n_samples) ++sbits;
  while (ibits < 32 && ((int64_t)1 << ibits) < nV) ++ibits;
  HCI_TRY(sort_keys(ctx, bp<uint64_t>(ctx->ss_draw), bp<uint64_t>(ctx->ss_draw2), m, sbits, ibits));
  HCI_TRY(ensure_buf(ctx, ctx->ss_run, (size_t)m * (8 + 8 + 8 + 4 + 4) + (size_t)(n_samples + 1) * 8));
  int64_t* flag = bp<int64_t>(ctx->ss_run);
  int64_t* pos = flag + m;
  int64_t* d_start = pos + m;
  int32_t* d_idx = reinterpret_cast<int32_t*>(d_start + m);
  int32_t* d_s = d_idx + m;
  int64_t* seg = reinterpret_cast<int64_t*>(d_s + m);
  int64_t* ndist_dev = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 48);
  HCI_LAUNCH(k_run_first, grid_for(m, 256, ctx->nsm * 8), 256, 0, st)(dk, m, flag);
  HCI_TRY(scan_i64(ctx, flag, pos, m, ndist_dev));
  HCI_LAUNCH(k_ss_compact, grid_for(m, 256, ctx->nsm * 8), 256, 0, st)(dk, m, flag, pos, d_idx, d_s, d_start);
  int64_t ndist = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&ndist, ndist_dev, 8, cudaMemcpyDeviceToHost, st));
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  HCI_LAUNCH(k_ss_seg, 1, 256, 0, st)(d_s, ndist, n_samples, seg);
  std::vector<int64_t> seg_h((size_t)n_samples + 1);
  HCI_CUDA(ctx, cudaMemcpyAsync(seg_h.data(), seg, (size_t)(n_samples + 1) * 8, cudaMemcpyDeviceToHost, st));
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  int64_t maxsrc = 0;
  for (int s = 0; s < n_samples; ++s) maxsrc = std::max(maxsrc, seg_h[s + 1] - seg_h[s]);
  HCI_TRY(ensure_buf(ctx, ctx->ss_src, (size_t)maxsrc * 32));
  ulonglong2* sk = bp<ulonglong2>(ctx->ss_src);
  double* sc = reinterpret_cast<double*>(sk + maxsrc);
  double* sf = sc + maxsrc;
  // the reference of the diagonal elements (written by hci_pt2 above)
  WalkArgs A;
  HCI_TRY(pt_walk_args(ctx, A, reinterpret_cast<const uint64_t*>(sk), sc, 0, eps2));
  const size_t nref = 1 + 2 * (size_t)n + 4 * (size_t)n * n;
  double* ref = bp<double>(ctx->p2_ref);
  double* part = ref + nref;
  double* dsum = part + PT2_SUM_BLOCKS;
  const int64_t per = max_pairs > 0 ? max_pairs : ((int64_t)1 << 28);
  const ulonglong2* Vk = reinterpret_cast<const ulonglong2*>(keys);
  const size_t smref = nref * 8;
  HCI_CUDA(ctx, cudaFuncSetAttribute(k_ss_terms, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smref));
  HCI_TRY(ensure_buf(ctx, ctx->s_cand, (size_t)4096 * 16));
  HCI_TRY(ensure_buf(ctx, ctx->p2_vals, (size_t)4096 * 8));
  std::vector<double> est((size_t)n_samples * 2, 0.0);
  // one hash class of one sample's targets: walk (again with a larger
  // buffer if it was too small), sort, estimate, sum
  auto run_class = [&](int s, int npart, int pc, int64_t* m_out) -> hci_status {
    A.npart = npart;
    A.part = pc;
    int64_t mp = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
      A.out = bp<ulonglong2>(ctx->s_cand);
      A.vals = bp<double>(ctx->p2_vals);
      A.cap = (int64_t)std::min(ctx->s_cand.bytes / 16, ctx->p2_vals.bytes / 8);
      HCI_TRY(ensure_buf(ctx, ctx->p2_src, (size_t)A.cap * 4));
      A.srcs = bp<int32_t>(ctx->p2_src);
      HCI_TRY(run_walk(ctx, A, &mp));
      if (mp <= A.cap || (npart == 1 && mp > per)) break;
      HCI_TRY(ensure_buf(ctx, ctx->s_cand, (size_t)(mp + mp / 8 + 4096) * 16));
      HCI_TRY(ensure_buf(ctx, ctx->p2_vals, (size_t)(mp + mp / 8 + 4096) * 8));
    }
    *m_out = mp;
    if (npart == 1 && mp > per) return HCI_OK;
    if (mp > A.cap) return hci_fail(ctx, HCI_ERR_CUDA, "hci_pt2_stochastic: pair count changed between walks");
    if (mp == 0) return HCI_OK;
    HCI_TRY(ensure_buf(ctx, ctx->s_cand2, (size_t)mp * 16));
    HCI_TRY(ensure_buf(ctx, ctx->p2_vals2, (size_t)mp * 8));
    HCI_TRY(ensure_buf(ctx, ctx->p2_src2, (size_t)mp * 4));
    HCI_TRY(ensure_buf(ctx, ctx->p2_d, (size_t)mp * 8));
    HCI_TRY(sort_pairs(ctx, bp<uint64_t>(ctx->s_cand), bp<uint64_t>(ctx->s_cand2), bp<double>(ctx->p2_vals),
                       bp<double>(ctx->p2_vals2), bp<int32_t>(ctx->p2_src), bp<int32_t>(ctx->p2_src2), mp, n, n));
    double* ct = bp<double>(ctx->p2_vals2);
    double* cd = bp<double>(ctx->p2_d);
    HCI_LAUNCH(k_ss_terms, grid_for(mp, 256), 256, smref, st)(bp<ulonglong2>(ctx->s_cand), bp<double>(ctx->p2_vals),
                                                              bp<int32_t>(ctx->p2_src), mp, Vk, nV, sc, sf, eps2_det,
                                                              (double)nd, n, ref, A.ref_a, A.ref_b, e0, ct, cd);
    HCI_LAUNCH(k_sum_slices_d, PT2_SUM_BLOCKS, 256, 0, st)(ct, mp, part);
    HCI_LAUNCH(k_sum_parts_d, 1, 32, 0, st)(part, PT2_SUM_BLOCKS, dsum);
    HCI_LAUNCH(k_sum_slices_d, PT2_SUM_BLOCKS, 256, 0, st)(cd, mp, part);
    HCI_LAUNCH(k_sum_parts_d, 1, 32, 0, st)(part, PT2_SUM_BLOCKS, dsum + 1);
    HCI_CUDA(ctx, cudaGetLastError());
    double hs[2] = {0.0, 0.0};
    HCI_CUDA(ctx, cudaMemcpyAsync(hs, dsum, 16, cudaMemcpyDeviceToHost, st));
    HCI_CUDA(ctx, cudaStreamSynchronize(st));
    est[2 * (size_t)s] += hs[0];
    est[2 * (size_t)s + 1] += hs[1];
    return HCI_OK;
  };
  for (int s = 0; s < n_samples; ++s) {
    const int64_t j0 = seg_h[s], j1 = seg_h[s + 1];
    if (j1 <= j0) continue;
    HCI_LAUNCH(k_ss_gather, grid_for(j1 - j0, 256), 256, 0, st)(j0, j1, ndist, m, d_idx, d_start, Vk, c, W, total,
                                                                sk, sc, sf);
    A.nV = j1 - j0;
    int64_t tot_pairs = 0;
    HCI_TRY(run_class(s, 1, 0, &tot_pairs));
    if (tot_pairs > per) {
      const int64_t np64 = (tot_pairs + per - 1) / per;
      if (np64 > (1 << 20))
        return hci_fail(ctx, HCI_ERR_INVALID, "hci_pt2_stochastic: max_pairs too small for %lld pairs",
                        (long long)tot_pairs);
      const int npart = (int)np64;
      const int64_t cap = tot_pairs / npart + tot_pairs / (8 * (int64_t)npart) + 4096;
      HCI_TRY(ensure_buf(ctx, ctx->s_cand, (size_t)cap * 16));
      HCI_TRY(ensure_buf(ctx, ctx->p2_vals, (size_t)cap * 8));
      for (int pc = 0; pc < npart; ++pc) {
        int64_t mp = 0;
        HCI_TRY(run_class(s, npart, pc, &mp));
      }
    }
  }
  // Eq. (semistoc): E2^D plus the mean difference, and its standard error
  double mean = 0.0;
  for (int s = 0; s < n_samples; ++s) mean += est[2 * (size_t)s] - est[2 * (size_t)s + 1];
  mean /= n_samples;
  double var = 0.0;
  for (int s = 0; s < n_samples; ++s) {
    const double d = est[2 * (size_t)s] - est[2 * (size_t)s + 1] - mean;
    var += d * d;
  }
  result[0] = e2d + mean;
  result[1] = n_samples > 1 ? std::sqrt(var / (n_samples - 1) / n_samples) : 0.0;
  result[2] = e2d;
  if (sample_e2)
    for (size_t u = 0; u < est.size(); ++u) sample_e2[u] = est[u];
  return HCI_OK;
}
