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
// Both orientations (i,j) and (j,i) are stored in the graph, so the RDMs
// come out symmetric.  The diagonal part is reduced through the weighted
// occupation correlation M[sp][tq] = sum_i c_i^2 n_sp(i) n_tq(i).
#include "hci_internal.cuh"

namespace {

constexpr int R_WARPS = 8;

__device__ __forceinline__ void add2(double* r2, int n, int p, int q, int r, int s, double v) {
  atomicAdd(&r2[(((int64_t)p * n + q) * n + r) * n + s], v);
}

__global__ void __launch_bounds__(R_WARPS * 32) k_rdm_offdiag(int n, const ulonglong2* __restrict__ V, int64_t nV,
                                                              const double* __restrict__ c,
                                                              const int64_t* __restrict__ rowptr,
                                                              const int64_t* __restrict__ rowstart,
                                                              const int32_t* __restrict__ col, double* __restrict__ r1,
                                                              double* __restrict__ r2,
                                                              unsigned long long* __restrict__ queue) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long qi = 0;
    if (lane == 0) qi = atomicAdd(queue, 1ull);
    const int64_t i = (int64_t)__shfl_sync(0xffffffffu, qi, 0);
    if (i >= nV) break;
    const double ci = c[i];
    const ulonglong2 ki = V[i];
    const int64_t b = rowstart[i], e = b + (rowptr[i + 1] - rowptr[i]);
    for (int64_t k = b + lane; k < e; k += 32) {
      const int64_t j = col[k];
      const ulonglong2 kj = V[j];
      const double cc = ci * c[j];
      if (cc == 0.0) continue;
      const uint64_t xa = ki.x ^ kj.x, xb = ki.y ^ kj.y;
      const int da = __popcll(xa), db = __popcll(xb);
      if (da + db == 2) {
        // single a -> b in spin S
        const int S = da == 2 ? 0 : 1;
        const uint64_t sj = S == 0 ? kj.x : kj.y, oj = S == 0 ? kj.y : kj.x;
        const uint64_t x = S == 0 ? xa : xb;
        const int a = __ffsll((long long)(sj & x)) - 1;
        const int bb = __ffsll((long long)(x & ~sj)) - 1;
        const double w = cc * exc_phase(sj, a, bb);
        atomicAdd(&r1[a + (int64_t)bb * n], w);
        // spectators of the same spin (excluding a) and of the other spin
        uint64_t sp = sj & ~(1ull << a);
        while (sp) {
          const int kk = __ffsll((long long)sp) - 1;
          sp &= sp - 1;
          add2(r2, n, bb, a, kk, kk, w);
          add2(r2, n, kk, kk, bb, a, w);
          add2(r2, n, kk, a, bb, kk, -w);
          add2(r2, n, bb, kk, kk, a, -w);
        }
        uint64_t so = oj;
        while (so) {
          const int kk = __ffsll((long long)so) - 1;
          so &= so - 1;
          add2(r2, n, bb, a, kk, kk, w);
          add2(r2, n, kk, kk, bb, a, w);
        }
      } else if (da == 4 || db == 4) {
        const uint64_t sj = da == 4 ? kj.x : kj.y;
        const uint64_t x = da == 4 ? xa : xb;
        uint64_t holes = sj & x, parts = x & ~sj;
        const int a = __ffsll((long long)holes) - 1; holes &= holes - 1;
        const int bh = __ffsll((long long)holes) - 1;
        const int cp = __ffsll((long long)parts) - 1; parts &= parts - 1;
        const int d = __ffsll((long long)parts) - 1;
        const double s1 = exc_phase(sj, a, cp);
        const uint64_t t = sj ^ (1ull << a) ^ (1ull << cp);
        const double w = cc * s1 * exc_phase(t, bh, d);
        add2(r2, n, cp, a, d, bh, w);
        add2(r2, n, d, bh, cp, a, w);
        add2(r2, n, cp, bh, d, a, -w);
        add2(r2, n, d, a, cp, bh, -w);
      } else {
        // alpha a -> c, beta b -> d
        const int a = __ffsll((long long)(kj.x & xa)) - 1, cp = __ffsll((long long)(ki.x & xa)) - 1;
        const int bh = __ffsll((long long)(kj.y & xb)) - 1, d = __ffsll((long long)(ki.y & xb)) - 1;
        const double w = cc * exc_phase(kj.x, a, cp) * exc_phase(kj.y, bh, d);
        add2(r2, n, cp, a, d, bh, w);
        add2(r2, n, d, bh, cp, a, w);
      }
    }
  }
}

// M[s*n+p][t*n+q] = sum_i c_i^2 n_sp(i) n_tq(i), folded over the string
// groups of the cached graph.  One warp per alpha group g with weight
// W_g = sum_{i in g} c_i^2: the alpha-alpha block gets W_g for every pair of
// orbitals occupied in alpha_g, the alpha-beta block gets v_g[q] =
// sum_{i in g} c_i^2 n_q(beta_i) for every occupied p of alpha_g.  The
// beta-beta block is folded over the beta groups the same way.  Block
// partials live in shared memory and are added to M once per block.
__global__ void k_occ_groups(int n, const ulonglong2* __restrict__ V, const double* __restrict__ c,
                             const int64_t* __restrict__ ga, int64_t nua, const ulonglong2* __restrict__ bk,
                             const int32_t* __restrict__ permb, const int64_t* __restrict__ gb, int64_t nub,
                             double* __restrict__ M) {
  extern __shared__ double sm[];
  const int m = 2 * n;
  double* Ms = sm;                          // m*m
  double* vq = sm + m * m;                  // [warps][64]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* v = vq + wid * HCI_MAXORB;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) Ms[t] = 0.0;
  __syncthreads();
  const int64_t gw = (int64_t)blockIdx.x * nw + wid, nwarps = (int64_t)gridDim.x * nw;
  for (int64_t g = gw; g < nua; g += nwarps) {
    // v[q] = sum_{i in g} c_i^2 n_q(beta_i): lane q % 32 keeps v[q] in a
    // register, each 32-member chunk is reduced across the warp per orbital
    double v0 = 0.0, v1 = 0.0, W = 0.0;
    const int64_t b = ga[g], e = ga[g + 1];
    for (int64_t i0 = b; i0 < e; i0 += 32) {
      const int64_t i = i0 + lane;
      const double w = i < e ? c[i] * c[i] : 0.0;
      const uint64_t y = i < e ? V[i].y : 0ull;
      W += w;
      for (int q = 0; q < n; ++q) {
        double t = ((y >> q) & 1ull) ? w : 0.0;
        if (__any_sync(0xffffffffu, t != 0.0)) {
          for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (lane == (q & 31)) { if (q < 32) v0 += t; else v1 += t; }
        }
      }
    }
    for (int o = 16; o; o >>= 1) W += __shfl_xor_sync(0xffffffffu, W, o);
    v[lane] = v0;
    v[lane + 32] = v1;
    __syncwarp();
    const uint64_t a = V[b].x;
    for (int t = lane; t < n * n; t += 32) {
      const int p = t / n, q = t % n;
      if (!((a >> p) & 1ull)) continue;
      if ((a >> q) & 1ull) atomicAdd(&Ms[p * m + q], W);
      if (v[q] != 0.0) {
        atomicAdd(&Ms[p * m + n + q], v[q]);
        atomicAdd(&Ms[(n + q) * m + p], v[q]);
      }
    }
    __syncwarp();
  }
  for (int64_t g = gw; g < nub; g += nwarps) {
    double W = 0.0;
    const int64_t b = gb[g], e = gb[g + 1];
    for (int64_t k = b + lane; k < e; k += 32) {
      const double cv = c[permb[k]];
      W += cv * cv;
    }
    for (int o = 16; o; o >>= 1) W += __shfl_xor_sync(0xffffffffu, W, o);
    const uint64_t bb = bk[b].x;
    for (int t = lane; t < n * n; t += 32) {
      const int p = t / n, q = t % n;
      if (((bb >> p) & 1ull) && ((bb >> q) & 1ull)) atomicAdd(&Ms[(n + p) * m + n + q], W);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m * m; t += blockDim.x)
    if (Ms[t] != 0.0) atomicAdd(&M[t], Ms[t]);
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
  const size_t smem = (size_t)4 * n2 * 8 + 8 * HCI_MAXORB * 8;
  HCI_CUDA(ctx, cudaFuncSetAttribute(k_occ_groups, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     4 * 64 * 64 * 8 + 8 * HCI_MAXORB * 8));
  HCI_LAUNCH(k_occ_groups, 152, 256, smem, st)(n, V, c, bp<int64_t>(ctx->g_ga), ctx->graph.nua,
                                               bp<ulonglong2>(ctx->g_bkeys), bp<int32_t>(ctx->g_permb),
                                               bp<int64_t>(ctx->g_gb), ctx->graph.nub, M);
  HCI_LAUNCH(k_diag_rdm, grid_for((int64_t)n2, 256), 256, 0, st)(n, M, rdm1, rdm2);
  prof_toc(ctx, HCI_PH_RDM_DIAG);
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(bp<char>(ctx->s_counter) + 56);
  HCI_CUDA(ctx, cudaMemsetAsync(queue, 0, 8, st));
  HCI_LAUNCH(k_rdm_offdiag, 152 * 8, R_WARPS * 32, 0, st)(n, V, nV, c, bp<int64_t>(ctx->graph.rowptr),
                                                         bp<int64_t>(ctx->graph.rowstart),
                                                   bp<int32_t>(ctx->graph.col), rdm1, rdm2, queue);
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_RDM);
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  return HCI_OK;
}
