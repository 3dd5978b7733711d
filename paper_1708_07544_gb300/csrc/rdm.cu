// Spin-summed variational 1- and 2-RDMs accumulated over the connections of
// V (Sec. IV: the variational RDMs reuse the single/double connections of
// the Hamiltonian build; Gamma^{c,c} of Eq. vdedk2).
//
//   rdm1[p,q]     = sum_s  <a+_ps a_qs>
//   rdm2[p,q,r,s] = sum_st <a+_ps a+_rt a_st a_qs>
//
// For a connection D_i = phase * (excitation of D_j) with weight
// w = c_i c_j phase, the non-zero operator strings are:
//   single a->b (spin S), each spectator k occupied in D_j (spin T):
//     rdm1[b,a] += w; rdm2[b,a,k,k] += w; rdm2[k,k,b,a] += w;
//     if T == S: rdm2[k,a,b,k] -= w; rdm2[b,k,k,a] -= w
//   double a->c, b->d (holes a<b, particles c<d in one spin, or a->c alpha
//   and b->d beta): rdm2[c,a,d,b] += w; rdm2[d,b,c,a] += w;
//     same spin only: rdm2[c,b,d,a] -= w; rdm2[d,a,c,b] -= w
// One orientation of each connected pair is accumulated (the graph stores
// one, or both) and the other added as its transpose.  The diagonal part is
// reduced through the weighted
// occupation correlation M[sp][tq] = sum_i c_i^2 n_sp(i) n_tq(i), folded over
// the alpha and beta string groups of the graph.
#include "hci_internal.cuh"
#include "rdm_acc.cuh"

namespace {

constexpr int R_WARPS = 8;


// One warp per row from a queue.  One-orientation graphs: every stored entry
// is one orientation of a connected pair; both-orientation graphs: the
// entries with j > i are.
__global__ void __launch_bounds__(R_WARPS * 32) k_rdm_offdiag(int n, const ulonglong2* __restrict__ V, int64_t nV,
                                                              const double* __restrict__ c,
                                                              const int64_t* __restrict__ rowptr,
                                                              const int64_t* __restrict__ rowstart,
                                                              const __grid_constant__ SegTab T, int both, RdmAcc R,
                                                              unsigned long long* __restrict__ queue) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long qi = 0;
    if (lane == 0) qi = atomicAdd(queue, 1ull);
    const int64_t i = (int64_t)__shfl_sync(0xffffffffu, qi, 0);
    if (i >= nV) break;
    const double ci = c[i];
    if (ci == 0.0) continue;
    const ulonglong2 ki = V[i];
    const int64_t rs = rowstart[i], len = rowptr[i + 1] - rowptr[i];
    const int32_t* col = T.col[rs >> GRAPH_SEG_SHIFT] + (rs & GRAPH_SEG_MASK);
    for (int64_t k = lane; k < len; k += 32) {
      const int64_t j = col[k];
      if (both && j <= i) continue;
      const double cc = ci * c[j];
      if (cc == 0.0) continue;
      rdm_accumulate(R, n, ki, V[j], cc);
    }
  }
}

// Single-excitation spectator sums: Xt[b][a][k] over both spins,
// Xx[b][a][k] over the excitation's own spin (spectator k != a).
__device__ __forceinline__ double rdm_xt(const RdmAcc& R, int n, int b, int a, int k) {
  const int64_t ba = (int64_t)b * n + a;
  const double s = R.S1[ba] + R.S1[(int64_t)n * n + ba];
  const int occ = (int)((R.ref_a >> k) & 1ull) + (int)((R.ref_b >> k) & 1ull) - (k == a);
  return s * occ + R.Dt[ba * n + k];
}
__device__ __forceinline__ double rdm_xx(const RdmAcc& R, int n, int b, int a, int k) {
  const int64_t ba = (int64_t)b * n + a;
  const int oa = (int)((R.ref_a >> k) & 1ull) - (k == a), ob = (int)((R.ref_b >> k) & 1ull) - (k == a);
  return R.S1[ba] * oa + R.S1[(int64_t)n * n + ba] * ob + R.Dx[ba * n + k];
}
// the single-excitation terms of one orientation at (p,q,r,s)
__device__ __forceinline__ double rdm_single_terms(const RdmAcc& R, int n, int p, int q, int r, int s) {
  double v = 0.0;
  if (r == s) v += rdm_xt(R, n, p, q, r);
  if (p == q) v += rdm_xt(R, n, r, s, p);
  if (s == p) v -= rdm_xx(R, n, r, q, p);
  if (q == r) v -= rdm_xx(R, n, p, s, q);
  return v;
}

// rdm2 += Hh + single terms, rdm1 += S1 (the accumulated orientation), and
// with sym also their transposes (the other orientation of every pair)
__global__ void k_rdm_finish(int n, RdmAcc R, double* __restrict__ r1, double* __restrict__ r2, int sym) {
  const int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t % n), r = (int)((t / n) % n), q = (int)((t / n2) % n), p = (int)(t / (n2 * n));
    double v = R.Hh[t] + rdm_single_terms(R, n, p, q, r, s);
    if (sym) {
      const int64_t tt = (((int64_t)q * n + p) * n + s) * n + r;
      v += R.Hh[tt] + rdm_single_terms(R, n, q, p, s, r);
    }
    r2[t] += v;
    if (t < n2) {
      const int pp = (int)(t / n), qq = (int)(t % n);
      double w = R.S1[t] + R.S1[n2 + t];
      if (sym) w += R.S1[(int64_t)qq * n + pp] + R.S1[n2 + (int64_t)qq * n + pp];
      r1[t] += w;
    }
  }
}

// Transition density of screened perturbative pairs: <V[src[j]]| op |tgt[j]>
// with weight c[src[j]] d[j] (pairs with d = 0 skipped).
__global__ void k_rdm_pairs(int n, const ulonglong2* __restrict__ V, const double* __restrict__ c,
                            const ulonglong2* __restrict__ tgt, const int32_t* __restrict__ src,
                            const double* __restrict__ d, int64_t m, RdmAcc R) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const double dj = d[j];
    if (dj == 0.0) continue;
    const int32_t i = src[j];
    rdm_accumulate(R, n, V[i], tgt[j], c[i] * dj);
  }
}

// Occupation correlation sum_a w_a n(a) n(a)^T of the distinct targets (the
// first pair of each run of equal keys, w_a = d_a^2), over spin orbitals
// (alpha 0..n-1, beta n..2n-1), split about the aufbau occupations n_R:
// n(a) = n_R + delta_a, so acc = [W = sum w, u = sum w delta (2n),
// Q = sum w delta delta^T (2n x 2n)], block-local in shared memory first.
__global__ void k_dd_acc(int n, const ulonglong2* __restrict__ tgt, const double* __restrict__ d, int64_t m,
                         uint64_t ra, uint64_t rb, double* __restrict__ acc) {
  extern __shared__ double s_acc[];
  const int mm = 2 * n, nacc = 1 + mm + mm * mm;
  for (int t = threadIdx.x; t < nacc; t += blockDim.x) s_acc[t] = 0.0;
  __syncthreads();
  double* su = s_acc + 1;
  double* sq = s_acc + 1 + mm;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const ulonglong2 key = tgt[j];
    if (j > 0) {
      const ulonglong2 prev = tgt[j - 1];
      if (prev.x == key.x && prev.y == key.y) continue;
    }
    const double dj = d[j];
    if (dj == 0.0) continue;
    const double w = dj * dj;
    atomicAdd(&s_acc[0], w);
    const uint64_t da = key.x ^ ra, db = key.y ^ rb;
    for (int sk = 0; sk < 2; ++sk)
      for (uint64_t x = sk ? db : da; x; x &= x - 1) {
        const int ko = __ffsll((long long)x) - 1;
        const int k = sk * n + ko;
        const double dk = (((sk ? key.y : key.x) >> ko) & 1ull) ? 1.0 : -1.0;
        atomicAdd(&su[k], w * dk);
        for (int sl = 0; sl < 2; ++sl)
          for (uint64_t y = sl ? db : da; y; y &= y - 1) {
            const int lo = __ffsll((long long)y) - 1;
            const double dl = (((sl ? key.y : key.x) >> lo) & 1ull) ? 1.0 : -1.0;
            atomicAdd(&sq[k * mm + sl * n + lo], w * dk * dl);
          }
      }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nacc; t += blockDim.x)
    if (s_acc[t] != 0.0) atomicAdd(&acc[t], s_acc[t]);
}

// M = W n_R n_R^T + n_R u^T + u n_R^T + Q, the layout k_diag_rdm reads
__global__ void k_dd_matrix(int n, const double* __restrict__ acc, uint64_t ra, uint64_t rb, double* __restrict__ M) {
  const int mm = 2 * n;
  const double W = acc[0];
  const double* u = acc + 1;
  const double* Q = acc + 1 + mm;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < mm * mm; t += gridDim.x * blockDim.x) {
    const int k = t / mm, l = t % mm;
    const double nk = (k < n ? ((ra >> k) & 1ull) : ((rb >> (k - n)) & 1ull)) ? 1.0 : 0.0;
    const double nl = (l < n ? ((ra >> l) & 1ull) : ((rb >> (l - n)) & 1ull)) ? 1.0 : 0.0;
    M[t] = W * nk * nl + nk * u[l] + u[k] * nl + Q[t];
  }
}

// M[s*n+p][t*n+q] = sum_i c_i^2 n_sp(i) n_tq(i), folded over the string
// groups of the cached graph:
//  1. W_g = sum_{i in g} c_i^2 and v_g[q] = sum_{i in g} c_i^2 n_q(beta_i)
//     per alpha group g, Wb_h = sum_{i in h} c_i^2 per beta group h.
//  2. one thread per M entry and block per slice of groups: alpha-alpha
//     entries sum W_g over groups with p, q in alpha_g, alpha-beta entries
//     sum v_g[q] over groups with p in alpha_g, beta-beta entries sum Wb_h;
//     the slices' partial M are added in a fixed order.
// Step 1 cuts the determinants (alpha-major) and the beta-major positions
// into chunks of GW_CH consecutive members, one warp per chunk, so that a
// group holding a large share of the space is spread over many warps; each
// warp adds its partial sums to the groups it touched with atomics.
constexpr int GW_CH = 256;

__global__ void __launch_bounds__(256) k_group_weights(int n, const ulonglong2* __restrict__ V,
                                                       const double* __restrict__ c, const int32_t* __restrict__ ia,
                                                       int64_t nV, const int32_t* __restrict__ permb,
                                                       const int32_t* __restrict__ ib, double* __restrict__ Wa,
                                                       double* __restrict__ va, double* __restrict__ Wb) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nch = (nV + GW_CH - 1) / GW_CH;
  for (int64_t ch = warp; ch < 2 * nch; ch += nwarps) {
    const bool beta = ch >= nch;
    const int64_t i0 = (beta ? ch - nch : ch) * GW_CH;
    const int64_t i1 = i0 + GW_CH < nV ? i0 + GW_CH : nV;
    if (!beta) {
      // members in order; lane q accumulates orbitals q and q + 32
      // (broadcast loads, eight members fetched ahead)
      int g = ia[i0];
      double W = 0.0, v0 = 0.0, v1 = 0.0;
      for (int64_t ib0 = i0; ib0 < i1; ib0 += 8) {
        int gg[8];
        double cw[8];
        uint64_t yy[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int64_t i = ib0 + u;
          gg[u] = i < i1 ? ia[i] : g;
          cw[u] = i < i1 ? c[i] : 0.0;
          yy[u] = i < i1 ? V[i].y : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (gg[u] != g) {
            if (lane == 0) atomicAdd(&Wa[g], W);
            if (lane < n) atomicAdd(&va[(int64_t)g * n + lane], v0);
            if (lane + 32 < n) atomicAdd(&va[(int64_t)g * n + lane + 32], v1);
            g = gg[u];
            W = v0 = v1 = 0.0;
          }
          const double w = cw[u] * cw[u];
          W += w;
          if ((yy[u] >> lane) & 1ull) v0 += w;
          if ((yy[u] >> (lane + 32)) & 1ull) v1 += w;
        }
      }
      if (lane == 0) atomicAdd(&Wa[g], W);
      if (lane < n) atomicAdd(&va[(int64_t)g * n + lane], v0);
      if (lane + 32 < n) atomicAdd(&va[(int64_t)g * n + lane + 32], v1);
    } else {
      // one member per lane; groups are runs of consecutive positions, so a
      // sum over the lanes of equal group (shuffles down) leaves each run's
      // total in its first lane
      for (int64_t k0 = i0; k0 < i1; k0 += 32) {
        const int64_t k = k0 + lane;
        int h = -1;
        double w = 0.0;
        if (k < i1) {
          const int32_t d = permb[k];
          h = ib[d];
          w = c[d] * c[d];
        }
        for (int o = 1; o < 32; o <<= 1) {
          const double ow = __shfl_down_sync(0xffffffffu, w, o);
          const int oh = __shfl_down_sync(0xffffffffu, h, o);
          if (lane + o < 32 && oh == h) w += ow;
        }
        const int hp = __shfl_up_sync(0xffffffffu, h, 1);
        if (h >= 0 && (lane == 0 || hp != h)) atomicAdd(&Wb[h], w);
      }
    }
  }
}

constexpr int OCC_SLICES = 256;

__global__ void k_occ_sums(int n, const ulonglong2* __restrict__ V, const int64_t* __restrict__ ga, int64_t nua,
                           const ulonglong2* __restrict__ bk, const int64_t* __restrict__ gb, int64_t nub,
                           const double* __restrict__ Wa, const double* __restrict__ va,
                           const double* __restrict__ Wb, double* __restrict__ part) {
  // blockIdx.x: slice of groups, staged in shared memory in chunks; thread
  // t < 3n^2 owns one entry of the alpha-alpha (t < n^2), alpha-beta
  // (t < 2n^2) or beta-beta block
  constexpr int CH = 128;
  __shared__ uint64_t s_a[CH];
  __shared__ double s_w[CH];
  __shared__ double s_v[CH * HCI_MAXORB / 2];   // n <= 64: CH x n doubles staged in two halves
  const int m = 2 * n;
  const int64_t slice = blockIdx.x;
  const int64_t a0 = nua * slice / OCC_SLICES, a1 = nua * (slice + 1) / OCC_SLICES;
  const int64_t b0 = nub * slice / OCC_SLICES, b1 = nub * (slice + 1) / OCC_SLICES;
  const int nt = 3 * n * n;
  double acc[12];
  for (int r = 0; r < 12; ++r) acc[r] = 0.0;
  // alpha groups: strings, weights and v in chunks
  for (int64_t g0 = a0; g0 < a1; g0 += CH) {
    const int cnt = (int)(a1 - g0 < CH ? a1 - g0 : CH);
    for (int half = 0; half < 2; ++half) {
      const int q0 = half * (n / 2), q1 = half == 0 ? n / 2 : n;
      const int nq = q1 - q0;
      __syncthreads();
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        s_a[t] = V[ga[g0 + t]].x;
        s_w[t] = Wa[g0 + t];
      }
      for (int t = threadIdx.x; t < cnt * nq; t += blockDim.x) {
        const int gi = t / nq, qq = t % nq;
        s_v[gi * nq + qq] = va[(g0 + gi) * n + q0 + qq];
      }
      __syncthreads();
      int r = 0;
      for (int t = threadIdx.x; t < nt; t += blockDim.x, ++r) {
        if (t < n * n) {
          if (half) continue;
          const int p = t / n, q = t % n;
          double a = 0.0;
          for (int gi = 0; gi < cnt; ++gi) {
            const uint64_t x = s_a[gi];
            if (((x >> p) & 1ull) && ((x >> q) & 1ull)) a += s_w[gi];
          }
          acc[r] += a;
        } else if (t < 2 * n * n) {
          const int u = t - n * n, p = u / n, q = u % n;
          if (q < q0 || q >= q1) continue;
          double a = 0.0;
          for (int gi = 0; gi < cnt; ++gi)
            if ((s_a[gi] >> p) & 1ull) a += s_v[gi * nq + (q - q0)];
          acc[r] += a;
        }
      }
    }
  }
  // beta groups
  for (int64_t h0 = b0; h0 < b1; h0 += CH) {
    const int cnt = (int)(b1 - h0 < CH ? b1 - h0 : CH);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      s_a[t] = bk[gb[h0 + t]].x;
      s_w[t] = Wb[h0 + t];
    }
    __syncthreads();
    int r = 0;
    for (int t = threadIdx.x; t < nt; t += blockDim.x, ++r) {
      if (t < 2 * n * n) continue;
      const int u = t - 2 * n * n, p = u / n, q = u % n;
      double a = 0.0;
      for (int gi = 0; gi < cnt; ++gi) {
        const uint64_t x = s_a[gi];
        if (((x >> p) & 1ull) && ((x >> q) & 1ull)) a += s_w[gi];
      }
      acc[r] += a;
    }
  }
  int r = 0;
  double* P = part + slice * (int64_t)m * m;
  for (int t = threadIdx.x; t < nt; t += blockDim.x, ++r) {
    if (t < n * n) {
      const int p = t / n, q = t % n;
      P[p * m + q] = acc[r];
    } else if (t < 2 * n * n) {
      const int u = t - n * n, p = u / n, q = u % n;
      P[p * m + n + q] = acc[r];
      P[(n + q) * m + p] = acc[r];
    } else {
      const int u = t - 2 * n * n, p = u / n, q = u % n;
      P[(n + p) * m + n + q] = acc[r];
    }
  }
}

__global__ void k_sum_slices(int mm, const double* __restrict__ part, double* __restrict__ M) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= mm) return;
  double s = 0.0;
  for (int k = 0; k < OCC_SLICES; ++k) s += part[(int64_t)k * mm + t];
  M[t] = s;
}

// diagonal contributions from M
__global__ void k_diag_rdm(int n, const double* __restrict__ M, double* __restrict__ r1, double* __restrict__ r2) {
  const int m = 2 * n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x) {
    const int p = t / n, q = t % n;
    double coul = 0.0;
    for (int s = 0; s < 2; ++s)
      for (int u = 0; u < 2; ++u)
        if (!(p == q && s == u)) coul += M[(s * n + p) * m + u * n + q];
    r2[(((int64_t)p * n + p) * n + q) * n + q] += coul;
    if (p != q) {
      double ex = M[p * m + q] + M[(n + p) * m + n + q];
      r2[(((int64_t)p * n + q) * n + q) * n + p] -= ex;
    } else {
      r1[p * n + p] += M[p * m + p] + M[(n + p) * m + n + p];
    }
  }
}

}  // namespace

extern "C" hci_status hci_rdm12(hci_ctx* ctx, const uint64_t* keys, int64_t nV, const double* c, double* rdm1,
                                double* rdm2) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_rdm12: null context");
  if (nV <= 0 || !keys || !c || !rdm1 || !rdm2)
    return hci_fail(ctx, HCI_ERR_INVALID, "hci_rdm12: empty space or null pointer");
  HCI_TRY(graph_ensure(ctx, keys, nV));
  const int n = ctx->n;
  cudaStream_t st = ctx->st;
  prof_tic(ctx, HCI_PH_RDM);
  const size_t n2 = (size_t)n * n, n4 = n2 * n2;
  HCI_CUDA(ctx, cudaMemsetAsync(rdm1, 0, n2 * 8, st));
  HCI_CUDA(ctx, cudaMemsetAsync(rdm2, 0, n4 * 8, st));
  HCI_TRY(ensure_buf(ctx, ctx->s_misc, (size_t)4 * n2 * 8 + 64));
  double* M = bp<double>(ctx->s_misc);
  HCI_CUDA(ctx, cudaMemsetAsync(M, 0, 4 * n2 * 8, st));
  prof_tic(ctx, HCI_PH_RDM_DIAG);
  const ulonglong2* V = bp<ulonglong2>(ctx->graph.keys);
  {
    const Graph& G = ctx->graph;
    const int64_t nua = G.nua, nub = G.nub;
    const size_t mm = (size_t)4 * n2;
    HCI_TRY(ensure_buf(ctx, ctx->s_rdmw, (size_t)(nua + nub + nua * n + 16) * 8 + (size_t)OCC_SLICES * mm * 8));
    double* Wa = bp<double>(ctx->s_rdmw);
    double* Wb = Wa + nua;
    double* va = Wb + nub;
    double* part = va + nua * n;
    HCI_CUDA(ctx, cudaMemsetAsync(Wa, 0, (size_t)(nua + nub + nua * n) * 8, st));
    HCI_LAUNCH(k_group_weights, grid_for(2 * ((nV + GW_CH - 1) / GW_CH) * 32, 256), 256, 0, st)(
        n, V, c, bp<int32_t>(ctx->g_ia), nV, bp<int32_t>(ctx->g_permb), bp<int32_t>(ctx->g_ib), Wa, va, Wb);
    HCI_LAUNCH(k_occ_sums, OCC_SLICES, 1024, 0, st)(n, V, bp<int64_t>(ctx->g_ga), nua, bp<ulonglong2>(ctx->g_bkeys),
                                                   bp<int64_t>(ctx->g_gb), nub, Wa, va, Wb, part);
    HCI_LAUNCH(k_sum_slices, (unsigned)((mm + 255) / 256), 256, 0, st)((int)mm, part, M);
  }
  HCI_LAUNCH(k_diag_rdm, grid_for((int64_t)n2, 256), 256, 0, st)(n, M, rdm1, rdm2);
  prof_toc(ctx, HCI_PH_RDM_DIAG);
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(bp<char>(ctx->s_counter) + 56);
  HCI_CUDA(ctx, cudaMemsetAsync(queue, 0, 8, st));
  // the connections are stored by internal id
  HCI_TRY(ensure_buf(ctx, ctx->d_perm, (size_t)nV * 8));
  double* ci = bp<double>(ctx->d_perm);
  HCI_TRY(to_internal(ctx, c, ci, 1));
  const size_t n3 = n2 * n;
  HCI_TRY(ensure_buf(ctx, ctx->s_rdmh, (n4 + 2 * n2 + 2 * n3) * 8));
  HCI_CUDA(ctx, cudaMemsetAsync(ctx->s_rdmh.p, 0, (n4 + 2 * n2 + 2 * n3) * 8, st));
  RdmAcc R;
  R.Hh = bp<double>(ctx->s_rdmh);
  R.S1 = R.Hh + n4;
  R.Dt = R.S1 + 2 * n2;
  R.Dx = R.Dt + n3;
  R.ref_a = ctx->na == 64 ? ~0ull : ((1ull << ctx->na) - 1ull);
  R.ref_b = ctx->nb == 64 ? ~0ull : ((1ull << ctx->nb) - 1ull);
  if (ctx->graph.direct)
    HCI_TRY(direct_rdm(ctx, ci, R));   // connections searched again, one orientation each
  else
    HCI_LAUNCH(k_rdm_offdiag, ctx->nsm * 8, R_WARPS * 32, 0, st)(n, bp<ulonglong2>(ctx->graph.keys_int), nV, ci,
                                                                 bp<int64_t>(ctx->graph.rowptr),
                                                                 bp<int64_t>(ctx->graph.rowstart), ctx->graph.tab(),
                                                                 ctx->graph.half ? 0 : 1, R, queue);
  HCI_LAUNCH(k_rdm_finish, grid_for((int64_t)n4, 256, ctx->nsm * 8), 256, 0, st)(n, R, rdm1, rdm2, 1);
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_RDM);
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  return HCI_OK;
}

namespace {
// <S^2> = -N (N - 4) / 4 - 1/2 sum_pq rdm2[p,q,q,p], from S^2 = S_z^2 +
// (S_+ S_- + S_- S_+) / 2 written with the spin-summed 2-RDM of hci_rdm12
__global__ void k_spin_square(const double* __restrict__ rdm2, int n, int nelec, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int p = t / n, q = t % n;
    s += rdm2[(((int64_t)p * n + q) * n + q) * n + p];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = -0.25 * nelec * (nelec - 4.0) - 0.5 * red[0];
}
}  // namespace

extern "C" hci_status hci_spin_square(hci_ctx* ctx, const double* rdm2, double* s2) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_spin_square: null context");
  if (!rdm2 || !s2) return hci_fail(ctx, HCI_ERR_INVALID, "hci_spin_square: null pointer");
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  double* d = reinterpret_cast<double*>(bp<char>(ctx->s_counter) + 32);
  HCI_LAUNCH(k_spin_square, 1, 256, 0, ctx->st)(rdm2, ctx->n, ctx->na + ctx->nb, d);
  HCI_CUDA(ctx, cudaGetLastError());
  HCI_CUDA(ctx, cudaMemcpyAsync(s2, d, 8, cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  return HCI_OK;
}

// Density matrices of the perturbative correction, accumulated over the
// hash classes of hci_pt2: begin (clear), pairs (once per class), finish.
static RdmAcc pt2_acc(hci_ctx* ctx) {
  const size_t n = (size_t)ctx->n, n2 = n * n, n4 = n2 * n2;
  RdmAcc R;
  R.Hh = bp<double>(ctx->s_rdmh);
  R.S1 = R.Hh + n4;
  R.Dt = R.S1 + 2 * n2;
  R.Dx = R.Dt + n2 * n;
  R.ref_a = ctx->na == 64 ? ~0ull : ((1ull << ctx->na) - 1ull);
  R.ref_b = ctx->nb == 64 ? ~0ull : ((1ull << ctx->nb) - 1ull);
  return R;
}

hci_status pt2_rdm_begin(hci_ctx* ctx) {
  const size_t n = (size_t)ctx->n, n2 = n * n, n4 = n2 * n2, m = 2 * n;
  HCI_TRY(ensure_buf(ctx, ctx->s_rdmh, (n4 + 2 * n2 + 2 * n2 * n) * 8));
  HCI_CUDA(ctx, cudaMemsetAsync(ctx->s_rdmh.p, 0, (n4 + 2 * n2 + 2 * n2 * n) * 8, ctx->st));
  HCI_TRY(ensure_buf(ctx, ctx->p2_dd, (1 + m + 2 * m * m) * 8));
  HCI_CUDA(ctx, cudaMemsetAsync(ctx->p2_dd.p, 0, (1 + m + 2 * m * m) * 8, ctx->st));
  return HCI_OK;
}

hci_status pt2_rdm_pairs(hci_ctx* ctx, const ulonglong2* V, const double* c, const ulonglong2* tgt, const int32_t* src,
                         const double* d, int64_t m) {
  if (m <= 0) return HCI_OK;
  const int n = ctx->n, mm = 2 * n;
  RdmAcc R = pt2_acc(ctx);
  HCI_LAUNCH(k_rdm_pairs, grid_for(m, 256), 256, 0, ctx->st)(n, V, c, tgt, src, d, m, R);
  const size_t sm = (size_t)(1 + mm + mm * mm) * 8;
  HCI_CUDA(ctx, cudaFuncSetAttribute(k_dd_acc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  HCI_LAUNCH(k_dd_acc, grid_for(m, 256, ctx->nsm * 2), 256, sm, ctx->st)(n, tgt, d, m, R.ref_a, R.ref_b,
                                                                     bp<double>(ctx->p2_dd));
  HCI_CUDA(ctx, cudaGetLastError());
  return HCI_OK;
}

hci_status pt2_rdm_finish(hci_ctx* ctx, double* r1dd, double* r2dd, double* r1dc, double* r2dc) {
  const int n = ctx->n, mm = 2 * n;
  const size_t n2 = (size_t)n * n, n4 = n2 * n2;
  cudaStream_t st = ctx->st;
  RdmAcc R = pt2_acc(ctx);
  HCI_CUDA(ctx, cudaMemsetAsync(r1dc, 0, n2 * 8, st));
  HCI_CUDA(ctx, cudaMemsetAsync(r2dc, 0, n4 * 8, st));
  HCI_LAUNCH(k_rdm_finish, grid_for((int64_t)n4, 256, ctx->nsm * 8), 256, 0, st)(n, R, r1dc, r2dc, 0);
  double* acc = bp<double>(ctx->p2_dd);
  double* M = acc + 1 + mm + mm * mm;
  HCI_LAUNCH(k_dd_matrix, grid_for((int64_t)mm * mm, 256), 256, 0, st)(n, acc, R.ref_a, R.ref_b, M);
  HCI_CUDA(ctx, cudaMemsetAsync(r1dd, 0, n2 * 8, st));
  HCI_CUDA(ctx, cudaMemsetAsync(r2dd, 0, n4 * 8, st));
  HCI_LAUNCH(k_diag_rdm, grid_for((int64_t)n2, 256), 256, 0, st)(n, M, r1dd, r2dd);
  HCI_CUDA(ctx, cudaGetLastError());
  return HCI_OK;
}
