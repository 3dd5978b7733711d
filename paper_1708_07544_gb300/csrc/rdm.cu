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
    const int64_t b = rowptr[i], e = rowptr[i + 1];
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

// M[s*n+p][t*n+q] += sum_i c_i^2 n_sp n_tq  (block-private in shared memory)
__global__ void k_occ_corr(int n, const ulonglong2* __restrict__ V, int64_t nV, const double* __restrict__ c,
                           double* __restrict__ M) {
  extern __shared__ double sm[];
  const int m = 2 * n;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) sm[t] = 0.0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += (int64_t)gridDim.x * blockDim.x) {
    const double w = c[i] * c[i];
    if (w == 0.0) continue;
    const ulonglong2 k = V[i];
    for (int s = 0; s < 2; ++s) {
      uint64_t x = s == 0 ? k.x : k.y;
      while (x) {
        const int p = __ffsll((long long)x) - 1;
        x &= x - 1;
        for (int t = 0; t < 2; ++t) {
          uint64_t y = t == 0 ? k.x : k.y;
          while (y) {
            const int q = __ffsll((long long)y) - 1;
            y &= y - 1;
            atomicAdd(&sm[(s * n + p) * m + t * n + q], w);
          }
        }
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < m * m; t += blockDim.x)
    if (sm[t] != 0.0) atomicAdd(&M[t], sm[t]);
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
  const ulonglong2* V = bp<ulonglong2>(ctx->graph.keys);
  const size_t smem = (size_t)4 * n2 * 8;
  HCI_CUDA(ctx, cudaFuncSetAttribute(k_occ_corr, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 64 * 64 * 8));
  HCI_LAUNCH(k_occ_corr, grid_for(nV, 256, 152 * 2), 256, smem, st)(n, V, nV, c, M);
  HCI_LAUNCH(k_diag_rdm, grid_for((int64_t)n2, 256), 256, 0, st)(n, M, rdm1, rdm2);
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  unsigned long long* queue = reinterpret_cast<unsigned long long*>(bp<char>(ctx->s_counter) + 56);
  HCI_CUDA(ctx, cudaMemsetAsync(queue, 0, 8, st));
  HCI_LAUNCH(k_rdm_offdiag, 152 * 8, R_WARPS * 32, 0, st)(n, V, nV, c, bp<int64_t>(ctx->graph.rowptr),
                                                   bp<int32_t>(ctx->graph.col), rdm1, rdm2, queue);
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_RDM);
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  return HCI_OK;
}
