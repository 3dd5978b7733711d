// Relaxed density matrices of the HCI energy E_var + E2 (Sec. III.A,
// Eq. lambda): the z-vector equation for the response of c, and the
// assembly of the density whose contraction with the integral derivatives
// gives dE/dkappa at a fixed variational space and a fixed set of screened
// perturbative pairs.
//
// With c the normalised lowest eigenvector of H on V, d_a the first-order
// coefficients and g = dE2/dc (hci_pt2), a change dH of the Hamiltonian
// changes E_var + E2 by
//   (1 - |d|^2) <c|dH|c> + sum_a d_a^2 <D_a|dH|D_a> + 2 <d|dH|c>' - <z|dH|c>
// where z solves (H - E0) z = P g with z orthogonal to c (P = 1 - c c^T):
// the last term is g . dc for the eigenvector response (H - E0) dc =
// -P dH c.  For a real symmetric dH the symmetric parts suffice, so
//   Gamma = (1 - |d|^2) Gamma(c) + Gamma^dd + Gamma^dc + (Gamma^dc)^T
//           - 1/4 [Gamma(z + c) - Gamma(z - c)].
#include <cmath>
#include <vector>

#include "hci_internal.cuh"

namespace {

constexpr int ZB = 256;
constexpr int ZBLOCKS = 1024;

// part[b] = sum over block b's contiguous slice of a_i b_i, in order
__global__ void k_zv_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                         double* __restrict__ part) {
  __shared__ double red[ZB];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < n ? lo + per : n;
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s = fma(a[i], b[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_zv_sum(const double* __restrict__ part, int np, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < np; ++b) s += part[b];
    *out = s;
  }
}

// y = x + a w
__global__ void k_zv_axpy(double* __restrict__ y, const double* __restrict__ x, double a,
                          const double* __restrict__ w, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] + a * w[i];
}

// t = r / max(diag - e0, 1e-8)
__global__ void k_zv_prec(const double* __restrict__ r, const double* __restrict__ diag, double e0,
                          double* __restrict__ t, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double m = diag[i] - e0;
    if (m < 1e-8) m = 1e-8;
    t[i] = r[i] / m;
  }
}

// out = (1 - dd) G(c) + Gdd + Gdc + Gdc^T - 1/4 (G(z+c) - G(z-c)), for the
// 2-RDM (n^4, transpose (p,q,r,s) -> (q,p,s,r)) and the 1-RDM (n^2)
__global__ void k_relaxed_combine(int n, double dd, const double* __restrict__ gc1, const double* __restrict__ gc2,
                                  const double* __restrict__ gdd1, const double* __restrict__ gdd2,
                                  const double* __restrict__ gdc1, const double* __restrict__ gdc2,
                                  const double* __restrict__ gp1, const double* __restrict__ gp2,
                                  const double* __restrict__ gm1, const double* __restrict__ gm2,
                                  double* __restrict__ out1, double* __restrict__ out2) {
  const int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t % n), r = (int)((t / n) % n), q = (int)((t / n2) % n), p = (int)(t / (n2 * n));
    const int64_t tt = (((int64_t)q * n + p) * n + s) * n + r;
    out2[t] = (1.0 - dd) * gc2[t] + gdd2[t] + gdc2[t] + gdc2[tt] - 0.25 * (gp2[t] - gm2[t]);
    if (t < n2) {
      const int pp = (int)(t / n), qq = (int)(t % n);
      out1[t] = (1.0 - dd) * gc1[t] + gdd1[t] + gdc1[t] + gdc1[(int64_t)qq * n + pp] - 0.25 * (gp1[t] - gm1[t]);
    }
  }
}

struct ZVec {
  hci_ctx* ctx;
  int64_t n;
  double* part;
  double* scal;
  hci_status dot(const double* a, const double* b, double* host) {
    HCI_LAUNCH(k_zv_dot, ZBLOCKS, ZB, 0, ctx->st)(a, b, n, part);
    HCI_LAUNCH(k_zv_sum, 1, 32, 0, ctx->st)(part, ZBLOCKS, scal);
    HCI_CUDA(ctx, cudaGetLastError());
    HCI_CUDA(ctx, cudaMemcpyAsync(host, scal, 8, cudaMemcpyDeviceToHost, ctx->st));
    HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
    return HCI_OK;
  }
  hci_status axpy(double* y, const double* x, double a, const double* w) {
    HCI_LAUNCH(k_zv_axpy, grid_for(n, ZB), ZB, 0, ctx->st)(y, x, a, w, n);
    HCI_CUDA(ctx, cudaGetLastError());
    return HCI_OK;
  }
  // v <- v - (c . v) c
  hci_status project(double* v, const double* c) {
    double cv = 0.0;
    HCI_TRY(dot(c, v, &cv));
    return axpy(v, v, -cv, c);
  }
};

}  // namespace

extern "C" hci_status hci_zvector(hci_ctx* ctx, const uint64_t* keys, int64_t nV, const double* c, double e0,
                                  const double* rhs, double* z, double tol, int maxit, int* iters) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_zvector: null context");
  if (nV <= 0 || !keys || !c || !rhs || !z) return hci_fail(ctx, HCI_ERR_INVALID, "hci_zvector: empty space or null");
  if (maxit < 1) return hci_fail(ctx, HCI_ERR_INVALID, "hci_zvector: maxit < 1");
  if (iters) *iters = 0;
  HCI_TRY(graph_ensure(ctx, keys, nV));
  cudaStream_t st = ctx->st;
  const int64_t n = nV;
  // c, b (right-hand side), x (solution), r, p, q, y work vectors in the
  // graph's internal order, then the reduction scratch
  HCI_TRY(ensure_buf(ctx, ctx->d_zv, (size_t)7 * n * 8 + (size_t)(ZBLOCKS + 1) * 8));
  double* vc = bp<double>(ctx->d_zv);
  double* vb = vc + n;
  double* vx = vb + n;
  double* vr = vx + n;
  double* vp = vr + n;
  double* vq = vp + n;
  double* vy = vq + n;
  ZVec Z{ctx, n, vy + n, vy + n + ZBLOCKS};
  const double* diag = bp<double>(ctx->graph.diag);
  HCI_TRY(to_internal(ctx, c, vc, 1));
  HCI_TRY(to_internal(ctx, rhs, vb, 1));
  HCI_CUDA(ctx, cudaMemsetAsync(vx, 0, (size_t)n * 8, st));
  // r = P b, y = P M^-1 r, p = y
  HCI_CUDA(ctx, cudaMemcpyAsync(vr, vb, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
  HCI_TRY(Z.project(vr, vc));
  HCI_LAUNCH(k_zv_prec, grid_for(n, ZB), ZB, 0, st)(vr, diag, e0, vy, n);
  HCI_TRY(Z.project(vy, vc));
  HCI_CUDA(ctx, cudaMemcpyAsync(vp, vy, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
  double rho = 0.0, rr = 0.0;
  HCI_TRY(Z.dot(vr, vy, &rho));
  HCI_TRY(Z.dot(vr, vr, &rr));
  int it = 0;
  bool converged = std::sqrt(rr) <= tol;
  for (; it < maxit && !converged; ++it) {
    // q = P (H - e0) p
    HCI_TRY(sigma_apply(ctx, vp, vq, 1));
    HCI_TRY(Z.axpy(vq, vq, -e0, vp));
    HCI_TRY(Z.project(vq, vc));
    double pq = 0.0;
    HCI_TRY(Z.dot(vp, vq, &pq));
    if (!(pq > 0.0) || !std::isfinite(pq))
      return hci_fail(ctx, HCI_ERR_CUDA, "hci_zvector: p (H - E0) p = %.3e is not positive", pq);
    const double alpha = rho / pq;
    HCI_TRY(Z.axpy(vx, vx, alpha, vp));
    HCI_TRY(Z.axpy(vr, vr, -alpha, vq));
    HCI_TRY(Z.dot(vr, vr, &rr));
    if (std::sqrt(rr) <= tol) {
      converged = true;
      ++it;
      break;
    }
    HCI_LAUNCH(k_zv_prec, grid_for(n, ZB), ZB, 0, st)(vr, diag, e0, vy, n);
    HCI_TRY(Z.project(vy, vc));
    double rho2 = 0.0;
    HCI_TRY(Z.dot(vr, vy, &rho2));
    const double beta = rho2 / rho;
    rho = rho2;
    HCI_TRY(Z.axpy(vp, vy, beta, vp));
  }
  // keep the solution orthogonal to c, back to the caller's order
  HCI_TRY(Z.project(vx, vc));
  HCI_TRY(to_sorted(ctx, vx, z, 1));
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  if (iters) *iters = it;
  if (!converged)
    return hci_fail(ctx, HCI_ERR_NOT_CONVERGED, "hci_zvector: residual %.3e > tol %.3e after %d iterations",
                    std::sqrt(rr), tol, it);
  return HCI_OK;
}

extern "C" hci_status hci_relaxed_rdm12(hci_ctx* ctx, double eps2, const uint64_t* keys, const double* c,
                                        int64_t nV, double e0, int64_t max_pairs, double zv_tol, int zv_maxit,
                                        double* e2, double* rdm1, double* rdm2) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_relaxed_rdm12: null context");
  if (nV <= 0 || !keys || !c || !e2 || !rdm1 || !rdm2)
    return hci_fail(ctx, HCI_ERR_INVALID, "hci_relaxed_rdm12: empty space or null pointer");
  const int n = ctx->n;
  const size_t n2 = (size_t)n * n, n4 = n2 * n2;
  cudaStream_t st = ctx->st;
  // six 1-/2-RDM pairs (Gamma^dd, Gamma^dc, G(c), G(z+c), G(z-c)) and g, z, z+-c
  HCI_TRY(ensure_buf(ctx, ctx->d_rel, (size_t)5 * (n2 + n4) * 8 + (size_t)4 * nV * 8));
  double* base = bp<double>(ctx->d_rel);
  double* g[10];
  for (int k = 0; k < 5; ++k) {
    g[2 * k] = base + (size_t)k * (n2 + n4);
    g[2 * k + 1] = g[2 * k] + n2;
  }
  double* vg = base + (size_t)5 * (n2 + n4);
  double* vz = vg + nV;
  double* vzp = vz + nV;
  double* vzm = vzp + nV;
  int64_t n_ext = 0;
  HCI_TRY(hci_pt2(ctx, eps2, keys, c, nV, e0, max_pairs, e2, &n_ext, g[0], g[1], g[2], g[3], vg));
  HCI_TRY(hci_zvector(ctx, keys, nV, c, e0, vg, vz, zv_tol, zv_maxit, nullptr));
  HCI_LAUNCH(k_zv_axpy, grid_for(nV, ZB), ZB, 0, st)(vzp, vz, 1.0, c, nV);
  HCI_LAUNCH(k_zv_axpy, grid_for(nV, ZB), ZB, 0, st)(vzm, vz, -1.0, c, nV);
  HCI_CUDA(ctx, cudaGetLastError());
  HCI_TRY(hci_rdm12(ctx, keys, nV, c, g[4], g[5]));
  HCI_TRY(hci_rdm12(ctx, keys, nV, vzp, g[6], g[7]));
  HCI_TRY(hci_rdm12(ctx, keys, nV, vzm, g[8], g[9]));
  // |d|^2 = tr Gamma^dd_1 / N
  std::vector<double> t1(n2);
  HCI_CUDA(ctx, cudaMemcpyAsync(t1.data(), g[0], n2 * 8, cudaMemcpyDeviceToHost, st));
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  double tr = 0.0;
  for (int p = 0; p < n; ++p) tr += t1[(size_t)p * n + p];
  const int N = ctx->na + ctx->nb;
  const double dd = N > 0 ? tr / N : 0.0;
  HCI_LAUNCH(k_relaxed_combine, grid_for((int64_t)n4, ZB, ctx->nsm * 8), ZB, 0, st)(
      n, dd, g[4], g[5], g[0], g[1], g[2], g[3], g[6], g[7], g[8], g[9], rdm1, rdm2);
  HCI_CUDA(ctx, cudaGetLastError());
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  return HCI_OK;
}
