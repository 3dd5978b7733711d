// The variational stage of HCI end to end (Sec. II.A, Fig. 1a):
// V^0 = {aufbau determinant}, c^0 = [1]; repeat
//   C^mu = selection(V^mu, c^mu, eps1); stop if empty;
//   V^{mu+1} = V^mu + C^mu (sorted merge, c padded with zeros);
//   c^{mu+1}, E^{mu+1} = Davidson on V^{mu+1} warm-started from the padded c.
#include "hci_internal.cuh"

namespace {
__global__ void k_aufbau(int na, int nb, ulonglong2* keys, double* c) {
  uint64_t a = na == 64 ? ~0ull : ((1ull << na) - 1ull);
  uint64_t b = nb == 64 ? ~0ull : ((1ull << nb) - 1ull);
  keys[0] = make_ulonglong2(a, b);
  c[0] = 1.0;
}
}  // namespace

extern "C" hci_status hci_solve(hci_ctx* ctx, double eps1, int max_iter, double dav_tol, int dav_maxit,
                                uint64_t* keys_out, double* c_out, int64_t cap, int64_t* nV_out, double* energy,
                                int* iters) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_solve: null context");
  if (!nV_out || !energy) return hci_fail(ctx, HCI_ERR_INVALID, "hci_solve: null output scalar");
  if (max_iter < 0 || dav_maxit < 1) return hci_fail(ctx, HCI_ERR_INVALID, "hci_solve: bad iteration limits");
  *nV_out = 0;
  if (iters) *iters = 0;
  cudaStream_t st = ctx->st;
  HCI_TRY(hci_build_lists(ctx));
  // two ping-pong spaces and a buffer for the new determinants
  DevBuf kb[2], cb[2], nk;
  auto cleanup = [&]() {
    for (int i = 0; i < 2; ++i) { free_buf(st, kb[i]); free_buf(st, cb[i]); }
    free_buf(st, nk);
  };
  int cur = 0;
  int64_t nV = 1;
  hci_status s;
  if ((s = ensure_buf(ctx, kb[0], 16)) != HCI_OK || (s = ensure_buf(ctx, cb[0], 8)) != HCI_OK) { cleanup(); return s; }
  HCI_LAUNCH(k_aufbau, 1, 1, 0, st)(ctx->na, ctx->nb, bp<ulonglong2>(kb[0]), bp<double>(cb[0]));
  double e = 0.0;
  int dav_it = 0;
  s = hci_davidson(ctx, bp<uint64_t>(kb[0]), 1, bp<double>(cb[0]), &e, dav_tol, dav_maxit, &dav_it);
  if (s != HCI_OK) { cleanup(); return s; }
  int mu = 0;
  for (; mu < max_iter; ++mu) {
    int64_t ncap = nk.bytes / 16;
    int64_t nn = 0;
    s = hci_select(ctx, eps1, bp<uint64_t>(kb[cur]), bp<double>(cb[cur]), nV, bp<uint64_t>(nk), ncap, &nn);
    if (s == HCI_ERR_CAPACITY) {
      if ((s = ensure_buf(ctx, nk, (size_t)(nn + 1024) * 16)) != HCI_OK) { cleanup(); return s; }
      ncap = nk.bytes / 16;
      s = hci_select(ctx, eps1, bp<uint64_t>(kb[cur]), bp<double>(cb[cur]), nV, bp<uint64_t>(nk), ncap, &nn);
    }
    if (s != HCI_OK) { cleanup(); return s; }
    if (nn == 0) break;
    const int nxt = cur ^ 1;
    const int64_t nV2 = nV + nn;
    if ((s = ensure_buf(ctx, kb[nxt], (size_t)nV2 * 16)) != HCI_OK || (s = ensure_buf(ctx, cb[nxt], (size_t)nV2 * 8)) != HCI_OK) {
      cleanup();
      return s;
    }
    s = hci_merge(ctx, bp<uint64_t>(kb[cur]), bp<double>(cb[cur]), nV, bp<uint64_t>(nk), nn, bp<uint64_t>(kb[nxt]),
                  bp<double>(cb[nxt]));
    if (s != HCI_OK) { cleanup(); return s; }
    cur = nxt;
    nV = nV2;
    s = hci_davidson(ctx, bp<uint64_t>(kb[cur]), nV, bp<double>(cb[cur]), &e, dav_tol, dav_maxit, &dav_it);
    if (s != HCI_OK) { cleanup(); return s; }
  }
  if (iters) *iters = mu;
  *nV_out = nV;
  *energy = e;
  if (nV > cap) {
    cleanup();
    return hci_fail(ctx, HCI_ERR_CAPACITY, "hci_solve: %lld determinants exceed cap %lld", (long long)nV,
                    (long long)cap);
  }
  if (keys_out) HCI_CUDA(ctx, cudaMemcpyAsync(keys_out, kb[cur].p, (size_t)nV * 16, cudaMemcpyDeviceToDevice, st));
  if (c_out) HCI_CUDA(ctx, cudaMemcpyAsync(c_out, cb[cur].p, (size_t)nV * 8, cudaMemcpyDeviceToDevice, st));
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  cleanup();
  return HCI_OK;
}
