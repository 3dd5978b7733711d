// The variational stage of HCI end to end (Sec. II.A, Fig. 1a):
// V^0 = {aufbau determinant}, c^0 = [1]; repeat
//   C^mu = selection(V^mu, c^mu, eps1); stop if empty;
//   V^{mu+1} = V^mu + C^mu (sorted merge, c padded with zeros);
//   c^{mu+1}, E^{mu+1} = Davidson on V^{mu+1} warm-started from the padded c.
// hci_solve_batch runs many such solves concurrently, one context and one
// stream per in-flight instance, driven by a pool of host threads.
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "hci_internal.cuh"

namespace {
// c_eff[i] = max_r |c_r[i]|: the multi-state criterion max_r |H_ai c_i^(r)|
// is the single-state one with c_i replaced by c_eff[i]
__global__ void k_ceff(const double* __restrict__ c, int nroots, int64_t nV, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += (int64_t)gridDim.x * blockDim.x) {
    double m = 0.0;
    for (int r = 0; r < nroots; ++r) m = fmax(m, fabs(c[(int64_t)r * nV + i]));
    out[i] = m;
  }
}

__global__ void k_aufbau(int na, int nb, ulonglong2* keys, double* c) {
  uint64_t a = na == 64 ? ~0ull : ((1ull << na) - 1ull);
  uint64_t b = nb == 64 ? ~0ull : ((1ull << nb) - 1ull);
  keys[0] = make_ulonglong2(a, b);
  c[0] = 1.0;
}
}  // namespace

// The whole loop; on success the final space and vector are left in
// keys_res / c_res (owned by the caller, released with free_buf).  With
// keys0 given the loop resumes from (keys0, c0): the first selection is made
// from that state as it is, and its energy is only computed (by Davidson on
// it) when that selection is empty.
static hci_status solve_core(hci_ctx* ctx, double eps1, int max_iter, double dav_tol, int dav_maxit, DevBuf& keys_res,
                             DevBuf& c_res, int64_t* nV_out, double* energy, int* iters,
                             const uint64_t* keys0 = nullptr, const double* c0 = nullptr, int64_t nV0 = 0) {
  cudaStream_t st = ctx->st;
  HCI_TRY(hci_build_lists(ctx));
  DevBuf kb[2], cb[2], nk;
  auto cleanup = [&]() {
    for (int i = 0; i < 2; ++i) { free_buf(st, kb[i]); free_buf(st, cb[i]); }
    free_buf(st, nk);
  };
  int cur = 0;
  int64_t nV = keys0 ? nV0 : 1;
  hci_status s;
  if ((s = ensure_buf(ctx, kb[0], (size_t)nV * 16)) != HCI_OK || (s = ensure_buf(ctx, cb[0], (size_t)nV * 8)) != HCI_OK) {
    cleanup();
    return s;
  }
  double e = 0.0;
  int dav_it = 0;
  bool have_e = false;
  if (keys0) {
    cudaError_t ce = cudaMemcpyAsync(kb[0].p, keys0, (size_t)nV * 16, cudaMemcpyDeviceToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(cb[0].p, c0, (size_t)nV * 8, cudaMemcpyDeviceToDevice, st);
    if (ce != cudaSuccess) {
      cleanup();
      return hci_fail(ctx, HCI_ERR_CUDA, "hci_solve_from: %s", cudaGetErrorString(ce));
    }
  } else {
    HCI_LAUNCH(k_aufbau, 1, 1, 0, st)(ctx->na, ctx->nb, bp<ulonglong2>(kb[0]), bp<double>(cb[0]));
    // the first selection starts from c = [1] on the aufbau determinant; with
    // a spin parity that excludes it (odd, alpha = beta) V^0 holds no state
    if (ctx->spin_parity == 0) {
      s = hci_davidson(ctx, bp<uint64_t>(kb[0]), 1, bp<double>(cb[0]), &e, dav_tol, dav_maxit, &dav_it);
      if (s != HCI_OK) { cleanup(); return s; }
      have_e = true;
    }
  }
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
    have_e = false;
    const int nxt = cur ^ 1;
    const int64_t nV2 = nV + nn;
    if ((s = ensure_buf(ctx, kb[nxt], (size_t)nV2 * 16)) != HCI_OK ||
        (s = ensure_buf(ctx, cb[nxt], (size_t)nV2 * 8)) != HCI_OK) {
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
    have_e = true;
  }
  if (!have_e) {
    // resumed from a state whose space did not grow: its energy
    s = hci_davidson(ctx, bp<uint64_t>(kb[cur]), nV, bp<double>(cb[cur]), &e, dav_tol, dav_maxit, &dav_it);
    if (s != HCI_OK) { cleanup(); return s; }
  }
  if (iters) *iters = mu;
  *nV_out = nV;
  *energy = e;
  std::swap(keys_res, kb[cur]);
  std::swap(c_res, cb[cur]);
  cleanup();
  return HCI_OK;
}

static hci_status solve_entry(const char* name, hci_ctx* ctx, double eps1, int max_iter, double dav_tol,
                              int dav_maxit, uint64_t* keys_out, double* c_out, int64_t cap, int64_t* nV_out,
                              double* energy, int* iters, const uint64_t* keys0, const double* c0, int64_t nV0) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "%s: null context", name);
  if (!nV_out || !energy) return hci_fail(ctx, HCI_ERR_INVALID, "%s: null output scalar", name);
  if (max_iter < 0 || dav_maxit < 1) return hci_fail(ctx, HCI_ERR_INVALID, "%s: bad iteration limits", name);
  *nV_out = 0;
  if (iters) *iters = 0;
  cudaStream_t st = ctx->st;
  if (keys0) {
    if (nV0 < 1 || !c0) return hci_fail(ctx, HCI_ERR_INVALID, "%s: empty start space or null start vector", name);
    int ok = 0;
    HCI_TRY(check_sorted(ctx, keys0, nV0, &ok));
    if (!ok) return hci_fail(ctx, HCI_ERR_INVALID, "%s: start keys are not strictly ascending", name);
  }
  DevBuf kr, cr;
  int64_t nV = 0;
  double e = 0.0;
  hci_status s = solve_core(ctx, eps1, max_iter, dav_tol, dav_maxit, kr, cr, &nV, &e, iters, keys0, c0, nV0);
  if (s != HCI_OK) return s;
  *nV_out = nV;
  *energy = e;
  if (nV > cap) {
    free_buf(st, kr);
    free_buf(st, cr);
    return hci_fail(ctx, HCI_ERR_CAPACITY, "%s: %lld determinants exceed cap %lld", name, (long long)nV,
                    (long long)cap);
  }
  cudaError_t ce = cudaSuccess;
  if (keys_out) ce = cudaMemcpyAsync(keys_out, kr.p, (size_t)nV * 16, cudaMemcpyDeviceToDevice, st);
  if (ce == cudaSuccess && c_out) ce = cudaMemcpyAsync(c_out, cr.p, (size_t)nV * 8, cudaMemcpyDeviceToDevice, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  free_buf(st, kr);
  free_buf(st, cr);
  if (ce != cudaSuccess) return hci_fail(ctx, HCI_ERR_CUDA, "%s: %s", name, cudaGetErrorString(ce));
  return HCI_OK;
}

extern "C" hci_status hci_solve(hci_ctx* ctx, double eps1, int max_iter, double dav_tol, int dav_maxit,
                                uint64_t* keys_out, double* c_out, int64_t cap, int64_t* nV_out, double* energy,
                                int* iters) {
  return solve_entry("hci_solve", ctx, eps1, max_iter, dav_tol, dav_maxit, keys_out, c_out, cap, nV_out, energy, iters,
                     nullptr, nullptr, 0);
}

extern "C" hci_status hci_solve_from(hci_ctx* ctx, const uint64_t* keys0, const double* c0, int64_t nV0, double eps1,
                                     int max_iter, double dav_tol, int dav_maxit, uint64_t* keys_out, double* c_out,
                                     int64_t cap, int64_t* nV_out, double* energy, int* iters) {
  if (!keys0) return hci_fail(ctx, HCI_ERR_INVALID, "hci_solve_from: null start keys");
  return solve_entry("hci_solve_from", ctx, eps1, max_iter, dav_tol, dav_maxit, keys_out, c_out, cap, nV_out, energy,
                     iters, keys0, c0, nV0);
}

// Variational HCI for the nroots lowest states (Sec. II.A with the
// selection over all states): V^0 = {aufbau}, first selection from c = [1],
// then select with c_eff = max_r |c_r|, merge (every state padded with
// zeros), and the nroots lowest eigenpairs by deflated Davidson.
extern "C" hci_status hci_solve_roots(hci_ctx* ctx, int nroots, double eps1, int max_iter, double dav_tol,
                                      int dav_maxit, uint64_t* keys_out, double* c_out, int64_t cap, int64_t* nV_out,
                                      double* energies, int* iters) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_solve_roots: null context");
  if (!nV_out || !energies || nroots < 1) return hci_fail(ctx, HCI_ERR_INVALID, "hci_solve_roots: bad arguments");
  if (max_iter < 1 || dav_maxit < 1) return hci_fail(ctx, HCI_ERR_INVALID, "hci_solve_roots: bad iteration limits");
  *nV_out = 0;
  if (iters) *iters = 0;
  cudaStream_t st = ctx->st;
  HCI_TRY(hci_build_lists(ctx));
  DevBuf kb[2], cb[2], nk, ce;
  auto cleanup = [&]() {
    for (int i = 0; i < 2; ++i) { free_buf(st, kb[i]); free_buf(st, cb[i]); }
    free_buf(st, nk);
    free_buf(st, ce);
  };
  hci_status s;
  if ((s = ensure_buf(ctx, kb[0], 16)) != HCI_OK || (s = ensure_buf(ctx, ce, 8)) != HCI_OK) { cleanup(); return s; }
  HCI_LAUNCH(k_aufbau, 1, 1, 0, st)(ctx->na, ctx->nb, bp<ulonglong2>(kb[0]), bp<double>(ce));
  int cur = 0;
  int64_t nV = 1;
  int mu = 0;
  for (; mu < max_iter; ++mu) {
    if (mu > 0)
      HCI_LAUNCH(k_ceff, grid_for(nV, 256), 256, 0, st)(bp<double>(cb[cur]), nroots, nV, bp<double>(ce));
    int64_t ncap = nk.bytes / 16, nn = 0;
    s = hci_select(ctx, eps1, bp<uint64_t>(kb[cur]), bp<double>(ce), nV, bp<uint64_t>(nk), ncap, &nn);
    if (s == HCI_ERR_CAPACITY) {
      if ((s = ensure_buf(ctx, nk, (size_t)(nn + 1024) * 16)) != HCI_OK) { cleanup(); return s; }
      s = hci_select(ctx, eps1, bp<uint64_t>(kb[cur]), bp<double>(ce), nV, bp<uint64_t>(nk), nk.bytes / 16, &nn);
    }
    if (s != HCI_OK) { cleanup(); return s; }
    if (nn == 0) break;
    const int nxt = cur ^ 1;
    const int64_t nV2 = nV + nn;
    if ((s = ensure_buf(ctx, kb[nxt], (size_t)nV2 * 16)) != HCI_OK ||
        (s = ensure_buf(ctx, cb[nxt], (size_t)nV2 * nroots * 8)) != HCI_OK ||
        (s = ensure_buf(ctx, ce, (size_t)nV2 * 8)) != HCI_OK) {
      cleanup();
      return s;
    }
    for (int r = 0; r < nroots; ++r) {
      const double* cr = mu > 0 ? bp<double>(cb[cur]) + (int64_t)r * nV : nullptr;
      s = hci_merge(ctx, bp<uint64_t>(kb[cur]), cr, nV, bp<uint64_t>(nk), nn, bp<uint64_t>(kb[nxt]),
                    bp<double>(cb[nxt]) + (int64_t)r * nV2);
      if (s != HCI_OK) { cleanup(); return s; }
    }
    cur = nxt;
    nV = nV2;
    // while V holds fewer determinants than roots: all of its states (the
    // other rows of c stay zero)
    const int nr = nV < nroots ? (int)nV : nroots;
    s = hci_davidson_roots(ctx, bp<uint64_t>(kb[cur]), nV, nr, bp<double>(cb[cur]), energies, dav_tol, dav_maxit,
                           nullptr);
    if (s != HCI_OK) { cleanup(); return s; }
  }
  if (iters) *iters = mu;
  *nV_out = nV;
  if (mu == 0) { cleanup(); return hci_fail(ctx, HCI_ERR_INVALID, "hci_solve_roots: the first selection is empty"); }
  if (nV < nroots) {
    cleanup();
    return hci_fail(ctx, HCI_ERR_INVALID, "hci_solve_roots: the space ends with %lld < nroots determinants",
                    (long long)nV);
  }
  if (nV > cap) {
    cleanup();
    return hci_fail(ctx, HCI_ERR_CAPACITY, "hci_solve_roots: %lld determinants exceed cap %lld", (long long)nV,
                    (long long)cap);
  }
  cudaError_t e = cudaSuccess;
  if (keys_out) e = cudaMemcpyAsync(keys_out, kb[cur].p, (size_t)nV * 16, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && c_out) e = cudaMemcpyAsync(c_out, cb[cur].p, (size_t)nV * nroots * 8, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return hci_fail(ctx, HCI_ERR_CUDA, "hci_solve_roots: %s", cudaGetErrorString(e));
  return HCI_OK;
}

static std::mutex g_batch_mu;
static char g_batch_err[512] = {0};

extern "C" hci_status hci_solve_batch(int count, const int* norb, const int* nalpha, const int* nbeta,
                                      const double* const* h, const double* const* eri, const double* e_core,
                                      double eps1, int max_iter, double dav_tol, int dav_maxit, int nstreams,
                                      double* energies, int64_t* nV, double* const* rdm1, double* const* rdm2,
                                      int* status) {
  if (count < 0 || nstreams < 1) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_solve_batch: bad count or nstreams");
  if (count == 0) return HCI_OK;
  if (!norb || !nalpha || !nbeta || !h || !eri || !energies || !nV)
    return hci_fail(nullptr, HCI_ERR_INVALID, "hci_solve_batch: null argument array");
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return hci_fail(nullptr, HCI_ERR_CUDA, "hci_solve_batch: %s", cudaGetErrorString(ce));
  std::atomic<int> next{0};
  std::atomic<int> first_err{HCI_OK};
  g_batch_err[0] = 0;
  auto worker = [&]() {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      int z = HCI_OK;
      first_err.compare_exchange_strong(z, HCI_ERR_CUDA);
      return;
    }
    for (int k = next.fetch_add(1); k < count; k = next.fetch_add(1)) {
      hci_ctx* ctx = nullptr;
      hci_status s = hci_create(&ctx, norb[k], nalpha[k], nbeta[k], h[k], eri[k], e_core ? e_core[k] : 0.0, st);
      DevBuf kr, cr;
      int64_t n = 0;
      double e = 0.0;
      int it = 0;
      if (s == HCI_OK) s = solve_core(ctx, eps1, max_iter, dav_tol, dav_maxit, kr, cr, &n, &e, &it);
      if (s == HCI_OK && rdm1 && rdm2 && rdm1[k] && rdm2[k])
        s = hci_rdm12(ctx, bp<uint64_t>(kr), n, bp<double>(cr), rdm1[k], rdm2[k]);
      energies[k] = e;
      nV[k] = n;
      if (status) status[k] = s;
      if (s != HCI_OK) {
        int z = HCI_OK;
        if (first_err.compare_exchange_strong(z, s)) {
          std::lock_guard<std::mutex> lock(g_batch_mu);
          snprintf(g_batch_err, sizeof g_batch_err, "instance %d: %s", k, hci_last_error(ctx));
        }
      }
      if (ctx) {
        free_buf(st, kr);
        free_buf(st, cr);
        hci_destroy(ctx);
      }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  };
  const int nt = nstreams < count ? nstreams : count;
  std::vector<std::thread> pool;
  pool.reserve((size_t)nt);
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  const int err = first_err.load();
  if (err != HCI_OK) return hci_fail(nullptr, err, "hci_solve_batch: %s", g_batch_err);
  return HCI_OK;
}
