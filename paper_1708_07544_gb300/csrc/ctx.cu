// Context lifetime, integral tables and the heat-bath excitation lists.
#include <climits>
#include <cmath>
#include <cstdlib>
#include <new>

#include "hci_internal.cuh"

static thread_local char g_create_err[512] = {0};

int g_hci_nsm = 0;

int64_t hci_fail_alloc_env() {
  const char* v = getenv("HCI_FAIL_ALLOC_AFTER");
  if (!v || !*v) return -1;
  char* end = nullptr;
  const long long k = strtoll(v, &end, 10);
  return (end && *end == 0 && k >= 0) ? (int64_t)k : -1;
}

hci_status hci_fail(hci_ctx* ctx, hci_status code, const char* fmt, ...) {
  char* dst = ctx ? ctx->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

hci_status ensure_buf(hci_ctx* ctx, DevBuf& b, size_t bytes) {
  if (bytes <= b.bytes && b.p) return HCI_OK;
  if (ctx->fail_alloc_after >= 0) {
    if (ctx->fail_alloc_after == 0)
      return hci_fail(ctx, HCI_ERR_NOMEM, "device allocation of %zu bytes refused (injected by HCI_FAIL_ALLOC_AFTER)",
                      bytes);
    --ctx->fail_alloc_after;
  }
  if (b.p) {
    cudaFreeAsync(b.p, ctx->st);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t want = bytes < 256 ? 256 : bytes;
  want = (want + 255) & ~(size_t)255;
  cudaError_t e = cudaMallocAsync(&b.p, want, ctx->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return hci_fail(ctx, HCI_ERR_NOMEM, "device allocation of %zu bytes failed: %s", want,
                    cudaGetErrorString(e));
  }
  b.bytes = want;
  return HCI_OK;
}

void free_buf(cudaStream_t st, DevBuf& b) {
  if (b.p) cudaFreeAsync(b.p, st);
  b.p = nullptr;
  b.bytes = 0;
}

namespace {

// jk_same[p][r][k] = (pr|kk) - (pk|kr); j_opp[p][r][k] = (pr|kk)
__global__ void k_single_tables(int n, const double* __restrict__ eri, double* __restrict__ jk_same,
                                double* __restrict__ j_opp) {
  int64_t n3 = (int64_t)n * n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(t % n);
    int r = (int)((t / n) % n);
    int p = (int)(t / ((int64_t)n * n));
    double prkk = eri[(((int64_t)p * n + r) * n + k) * n + k];
    double pkkr = eri[(((int64_t)p * n + k) * n + k) * n + r];
    jk_same[t] = prkk - pkkr;
    j_opp[t] = prkk;
  }
}

// Upper bound of |H_ai| for a single p->r over all determinants:
// |h_pr| + sum_k |(pr|kk)-(pk|kr)| + sum_k |(pr|kk)|, padded for rounding.
__global__ void k_single_bound(int n, const double* __restrict__ h, const double* __restrict__ jk_same,
                               const double* __restrict__ j_opp, double* __restrict__ bound) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  int p = t / n, r = t % n;
  double b = fabs(h[p * n + r]);
  for (int k = 0; k < n; ++k) {
    b += fabs(jk_same[((int64_t)p * n + r) * n + k]);
    b += fabs(j_opp[((int64_t)p * n + r) * n + k]);
  }
  bound[t] = p == r ? 0.0 : b * (1.0 + 1e-10);
}

__device__ __forceinline__ void tri_decode(int t, int& lo, int& hi) {
  // t = hi*(hi-1)/2 + lo with lo < hi
  int h = (int)((1.0 + sqrt(1.0 + 8.0 * (double)t)) * 0.5);
  while (h * (h - 1) / 2 > t) --h;
  while ((h + 1) * h / 2 <= t) ++h;
  hi = h;
  lo = t - h * (h - 1) / 2;
}

__device__ __forceinline__ bool before(double ma, int ia, double mb, int ib) {
  return ma > mb || (ma == mb && ia < ib);
}

// One CTA per list: gather |v| for every target, bitonic sort (|v| desc,
// target index asc), write magnitudes and packed targets.
__global__ void k_build_lists(int n, const double* __restrict__ eri, int same, int L, int P,
                              double* __restrict__ mag_out, uint16_t* __restrict__ tgt_out) {
  extern __shared__ double sm_d[];
  double* m = sm_d;
  int* id = reinterpret_cast<int*>(m + P);
  const int list = blockIdx.x;
  int p, q;
  if (same) tri_decode(list, p, q);
  else { p = list / n; q = list % n; }
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    if (e < L) {
      int r, s;
      double v;
      if (same) {
        tri_decode(e, r, s);
        v = eri[(((int64_t)p * n + r) * n + q) * n + s] - eri[(((int64_t)p * n + s) * n + q) * n + r];
      } else {
        r = e / n;
        s = e % n;
        v = eri[(((int64_t)p * n + r) * n + q) * n + s];
      }
      m[e] = fabs(v);
      id[e] = e;
    } else {
      m[e] = -1.0;
      id[e] = INT_MAX;
    }
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          bool up = (i & k) == 0;   // ascending in "before" order
          double mi = m[i], ml = m[l];
          int ii = id[i], il = id[l];
          bool swap = up ? before(ml, il, mi, ii) : before(mi, ii, ml, il);
          if (swap) {
            m[i] = ml; m[l] = mi;
            id[i] = il; id[l] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < L; e += blockDim.x) {
    int src = id[e];
    int r, s;
    if (same) tri_decode(src, r, s);
    else { r = src / n; s = src % n; }
    mag_out[(int64_t)list * L + e] = m[e];
    tgt_out[(int64_t)list * L + e] = (uint16_t)(r | (s << 8));
  }
}

// f_ref[s][p][r] = h_pr + sum_{k occ in spin s of R} ((pr|kk) - (pk|kr))
//                       + sum_{k occ in the other spin of R} (pr|kk),  R = aufbau
__global__ void k_fref(int n, int na, int nb, const double* __restrict__ h, const double* __restrict__ jk_same,
                       const double* __restrict__ j_opp, double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * n * n) return;
  const int s = t / (n * n), p = (t / n) % n, r = t % n;
  const int ns = s == 0 ? na : nb, no = s == 0 ? nb : na;
  double v = h[p * n + r];
  for (int k = 0; k < n; ++k) {
    if (k < ns) v += jk_same[((int64_t)p * n + r) * n + k];
    if (k < no) v += j_opp[((int64_t)p * n + r) * n + k];
  }
  out[t] = v;
}

__global__ void k_gather_first(const double* __restrict__ mag, int nlists, int L, double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nlists) out[t] = mag[(int64_t)t * L];
}

__global__ void k_max_first(const double* __restrict__ mag, int nlists, int L, double* out) {
  double m = 0.0;
  for (int i = threadIdx.x; i < nlists; i += blockDim.x) m = fmax(m, mag[(int64_t)i * L]);
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double w[32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, w[k]);
    *out = r;
  }
}

__global__ void k_max_vec(const double* __restrict__ v, int n, double* out) {
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double w[32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, w[k]);
    *out = r;
  }
}

int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

extern "C" hci_status hci_create(hci_ctx** out, int norb, int nalpha, int nbeta, const double* h,
                                 const double* eri, double e_core, void* stream) {
  if (!out) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_create: out is NULL");
  *out = nullptr;
  if (norb < 1 || norb > HCI_MAXORB)
    return hci_fail(nullptr, HCI_ERR_INVALID, "hci_create: norb=%d outside [1,64]", norb);
  if (nalpha < 0 || nbeta < 0 || nalpha > norb || nbeta > norb)
    return hci_fail(nullptr, HCI_ERR_INVALID, "hci_create: nalpha=%d nbeta=%d invalid for norb=%d", nalpha,
                    nbeta, norb);
  if (!h || !eri) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_create: null integrals");
  hci_ctx* ctx = new (std::nothrow) hci_ctx();
  if (!ctx) return hci_fail(nullptr, HCI_ERR_NOMEM, "hci_create: host allocation failed");
  {
    // Workspaces come from the device's default stream-ordered pool; keep
    // freed memory in the pool (instead of unmapping it at every
    // synchronisation) so that a solve per orbital iteration reuses it.
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  }
  ctx->fail_alloc_after = hci_fail_alloc_env();
  {
    const char* v = getenv("HCI_SIGMA_HALF_PASSES");
    ctx->half_passes = (v && (v[0] == '1' || v[0] == '2') && v[1] == 0) ? v[0] - '0' : 0;
  }
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0) {
      ctx->nsm = nsm;
      g_hci_nsm = nsm;
    } else {
      ctx->nsm = hci_nsm();
    }
    size_t fr = 0, tot = 0;
    ctx->mem_total = cudaMemGetInfo(&fr, &tot) == cudaSuccess ? tot : ((size_t)64 << 30);
    int l2 = 0;
    ctx->l2_bytes = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess && l2 > 0
                        ? (size_t)l2 : ((size_t)126 << 20);
    cudaGetLastError();
  }
  ctx->n = norb;
  ctx->na = nalpha;
  ctx->nb = nbeta;
  ctx->ecore = e_core;
  ctx->st = (cudaStream_t)stream;
  const size_t n = (size_t)norb;
  hci_status s = HCI_OK;
  if ((s = ensure_buf(ctx, ctx->h, n * n * 8)) != HCI_OK ||
      (s = ensure_buf(ctx, ctx->eri, n * n * n * n * 8)) != HCI_OK ||
      (s = ensure_buf(ctx, ctx->jk_same, n * n * n * 8)) != HCI_OK ||
      (s = ensure_buf(ctx, ctx->j_opp, n * n * n * 8)) != HCI_OK ||
      (s = ensure_buf(ctx, ctx->lists.single_bound, n * n * 8)) != HCI_OK ||
      (s = ensure_buf(ctx, ctx->lists.f_ref, 2 * n * n * 8)) != HCI_OK) {
    snprintf(g_create_err, sizeof g_create_err, "%s", ctx->err);
    hci_destroy(ctx);
    return s;
  }
  cudaError_t e = cudaMemcpyAsync(ctx->h.p, h, n * n * 8, cudaMemcpyDeviceToDevice, ctx->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->eri.p, eri, n * n * n * n * 8, cudaMemcpyDeviceToDevice, ctx->st);
  if (e == cudaSuccess) {
    HCI_LAUNCH(k_single_tables, grid_for((int64_t)(n * n * n), 256), 256, 0, ctx->st)(
        norb, bp<double>(ctx->eri), bp<double>(ctx->jk_same), bp<double>(ctx->j_opp));
    HCI_LAUNCH(k_single_bound, (unsigned)((n * n + 255) / 256), 256, 0, ctx->st)(
        norb, bp<double>(ctx->h), bp<double>(ctx->jk_same), bp<double>(ctx->j_opp),
        bp<double>(ctx->lists.single_bound));
    HCI_LAUNCH(k_fref, (unsigned)((2 * n * n + 255) / 256), 256, 0, ctx->st)(
        norb, ctx->na, ctx->nb, bp<double>(ctx->h), bp<double>(ctx->jk_same), bp<double>(ctx->j_opp),
        bp<double>(ctx->lists.f_ref));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) {
    snprintf(g_create_err, sizeof g_create_err, "hci_create: %s", cudaGetErrorString(e));
    hci_destroy(ctx);
    return HCI_ERR_CUDA;
  }
  *out = ctx;
  return HCI_OK;
}

extern "C" hci_status hci_destroy(hci_ctx* ctx) {
  if (!ctx) return HCI_OK;
  cudaStream_t st = ctx->st;
  DevBuf* bufs[] = {&ctx->h, &ctx->eri, &ctx->jk_same, &ctx->j_opp, &ctx->lists.opp_mag, &ctx->lists.opp_tgt,
                    &ctx->lists.list_max, &ctx->lists.f_ref, &ctx->s_items,
                    &ctx->lists.same_mag, &ctx->lists.same_tgt, &ctx->lists.single_bound,
                    &ctx->graph.rowptr, &ctx->graph.rowstart, &ctx->graph.diag, &ctx->graph.keys,
                    &ctx->s_cand, &ctx->s_cand2, &ctx->s_flags, &ctx->s_scan, &ctx->s_misc, &ctx->s_counter,
                    &ctx->s_hist, &ctx->g_ua, &ctx->g_ga, &ctx->g_ia, &ctx->g_ub, &ctx->g_gb, &ctx->g_ib,
                    &ctx->g_permb, &ctx->g_bkeys, &ctx->g_bkeys2, &ctx->g_nbr_ptr, &ctx->g_nbr, &ctx->g_cnt,
                    &ctx->d_vb, &ctx->d_wb, &ctx->d_diag, &ctx->d_small, &ctx->d_part,
                    &ctx->g_bnbr_ptr, &ctx->g_bnbr, &ctx->g_costa, &ctx->g_costb, &ctx->s_walkstat,
                    &ctx->g_htab, &ctx->g_hval, &ctx->g_nscr, &ctx->s_rdmw, &ctx->g_posb, &ctx->g_vb, &ctx->g_ba,
                    &ctx->inc.pos_old, &ctx->inc.mark, &ctx->inc.flag, &ctx->inc.newrows, &ctx->inc.rpN,
                    &ctx->inc.cnt, &ctx->inc.keys_old, &ctx->inc.s2i_old, &ctx->inc.grow,
                    &ctx->inc.colN, &ctx->inc.valN, &ctx->inc.hist, &ctx->inc.tbase, &ctx->inc.T, &ctx->inc.T2,
                    &ctx->inc.tstart, &ctx->inc.len, &ctx->inc.rp_old, &ctx->inc.col_old, &ctx->inc.val_old,
                    &ctx->inc.len_old, &ctx->inc.cap_old, &ctx->graph.rowlen, &ctx->graph.rowcap,
                    &ctx->graph.keys_int, &ctx->graph.s2i, &ctx->graph.i2s,
                    &ctx->d_perm, &ctx->s_rdmh, &ctx->inc.scr, &ctx->inc.stage,
                    &ctx->inc.roff, &ctx->inc.ctl, &ctx->inc.left, &ctx->inc.samp,
                    &ctx->p2_vals, &ctx->p2_vals2, &ctx->p2_ref,
                    &ctx->p2_src, &ctx->p2_src2, &ctx->p2_d, &ctx->p2_dd,
                    &ctx->d_zv, &ctx->d_rel, &ctx->d_lock, &ctx->d_partner, &ctx->dkeep.Q, &ctx->dkeep.W, &ctx->ss_w, &ctx->ss_draw,
                    &ctx->ss_draw2, &ctx->ss_run, &ctx->ss_src};
  for (int k = 0; k < GRAPH_MAXSEG; ++k) {
    free_buf(st, ctx->graph.seg_col[k]);
    free_buf(st, ctx->graph.seg_val[k]);
  }
  for (DevBuf* b : bufs) free_buf(st, *b);
  prof_release(ctx);
  cudaStreamSynchronize(st);
  delete ctx;
  return HCI_OK;
}

extern "C" const char* hci_last_error(const hci_ctx* ctx) { return ctx ? ctx->err : g_create_err; }

extern "C" hci_status hci_build_lists(hci_ctx* ctx) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_build_lists: null context");
  Lists& L = ctx->lists;
  if (L.built) return HCI_OK;
  const int n = ctx->n;
  prof_tic(ctx, HCI_PH_LISTS);
  L.n = n;
  L.len_opp = n * n;
  L.npair_same = n * (n - 1) / 2;
  L.len_same = L.npair_same;
  HCI_TRY(ensure_buf(ctx, L.opp_mag, (size_t)n * n * L.len_opp * 8));
  HCI_TRY(ensure_buf(ctx, L.opp_tgt, (size_t)n * n * L.len_opp * 2));
  if (L.npair_same > 0) {
    HCI_TRY(ensure_buf(ctx, L.same_mag, (size_t)L.npair_same * L.len_same * 8));
    HCI_TRY(ensure_buf(ctx, L.same_tgt, (size_t)L.npair_same * L.len_same * 2));
  }
  {
    int P = next_pow2(L.len_opp);
    size_t smem = (size_t)P * 12;
    HCI_CUDA(ctx, cudaFuncSetAttribute(k_build_lists, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    HCI_LAUNCH(k_build_lists, n * n, 1024, smem, ctx->st)(n, bp<double>(ctx->eri), 0, L.len_opp, P,
                                                  bp<double>(L.opp_mag), bp<uint16_t>(L.opp_tgt));
    HCI_CUDA(ctx, cudaGetLastError());
  }
  if (L.npair_same > 0) {
    int P = next_pow2(L.len_same);
    size_t smem = (size_t)P * 12;
    HCI_LAUNCH(k_build_lists, L.npair_same, 1024, smem, ctx->st)(n, bp<double>(ctx->eri), 1, L.len_same, P,
                                                         bp<double>(L.same_mag), bp<uint16_t>(L.same_tgt));
    HCI_CUDA(ctx, cudaGetLastError());
  }
  HCI_TRY(ensure_buf(ctx, L.list_max, (size_t)(n * n + L.npair_same + 1) * 8));
  HCI_LAUNCH(k_gather_first, (n * n + 255) / 256, 256, 0, ctx->st)(bp<double>(L.opp_mag), n * n, L.len_opp,
                                                                  bp<double>(L.list_max));
  if (L.npair_same > 0)
    HCI_LAUNCH(k_gather_first, (L.npair_same + 255) / 256, 256, 0, ctx->st)(
        bp<double>(L.same_mag), L.npair_same, L.len_same, bp<double>(L.list_max) + n * n);
  HCI_TRY(ensure_buf(ctx, ctx->s_misc, 64));
  double* dm = bp<double>(ctx->s_misc);
  HCI_CUDA(ctx, cudaMemsetAsync(dm, 0, 64, ctx->st));
  HCI_LAUNCH(k_max_first, 1, 1024, 0, ctx->st)(bp<double>(L.opp_mag), n * n, L.len_opp, dm + 0);
  if (L.npair_same > 0)
    HCI_LAUNCH(k_max_first, 1, 1024, 0, ctx->st)(bp<double>(L.same_mag), L.npair_same, L.len_same, dm + 1);
  HCI_LAUNCH(k_max_vec, 1, 1024, 0, ctx->st)(bp<double>(L.single_bound), n * n, dm + 2);
  HCI_CUDA(ctx, cudaGetLastError());
  double hm[3];
  HCI_CUDA(ctx, cudaMemcpyAsync(hm, dm, 24, cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  L.max_opp = hm[0];
  L.max_same = hm[1];
  L.max_single = hm[2];
  L.built = true;
  prof_toc(ctx, HCI_PH_LISTS);
  return HCI_OK;
}

extern "C" hci_status hci_set_sigma_mode(hci_ctx* ctx, int mode, int64_t graph_budget) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_set_sigma_mode: null context");
  if (mode != HCI_SIGMA_AUTO && mode != HCI_SIGMA_STORED && mode != HCI_SIGMA_DIRECT && mode != HCI_SIGMA_HALF)
    return hci_fail(ctx, HCI_ERR_INVALID, "hci_set_sigma_mode: unknown mode %d", mode);
  if (graph_budget < 0) return hci_fail(ctx, HCI_ERR_INVALID, "hci_set_sigma_mode: negative budget");
  ctx->sigma_mode = mode;
  ctx->graph_budget = graph_budget;
  ctx->direct_fallback = false;
  ctx->half_fallback = false;
  ctx->graph.valid = false;
  return HCI_OK;
}

extern "C" hci_status hci_stats(const hci_ctx* ctx, int64_t* out, int nout) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_stats: null context");
  if (nout < 0 || (nout > 0 && !out)) return HCI_ERR_INVALID;
  int64_t v[HCI_ST_COUNT];
  for (int k = 0; k < HCI_ST_COUNT; ++k) v[k] = ctx->st_counts[k];
  v[HCI_ST_GRAPH_NNZ] = ctx->graph.valid && ctx->graph.nnz > 0 ? ctx->graph.nnz : 0;
  v[HCI_ST_LAST_CANDIDATES] = ctx->last_candidates;
  v[HCI_ST_SIGMA_DIRECT] = ctx->graph.valid && ctx->graph.direct ? 1 : 0;
  v[HCI_ST_GRAPH_HALF] = ctx->graph.valid && !ctx->graph.direct && ctx->graph.half ? 1 : 0;
  for (int k = 0; k < nout && k < HCI_ST_COUNT; ++k) out[k] = v[k];
  for (int k = HCI_ST_COUNT; k < nout; ++k) out[k] = 0;
  return HCI_OK;
}

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------
std::atomic<long long> g_hci_launches{0};

static cudaEvent_t prof_event(hci_ctx* ctx) {
  if (!ctx->prof.pool.empty()) {
    cudaEvent_t e = ctx->prof.pool.back();
    ctx->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void prof_tic(hci_ctx* ctx, int phase) {
  if (!ctx->prof.on) return;
  cudaEvent_t e = prof_event(ctx);
  if (!e) return;
  cudaEventRecord(e, ctx->st);
  ctx->prof.open[phase] = e;
}

void prof_toc(hci_ctx* ctx, int phase) {
  if (!ctx->prof.on || !ctx->prof.open[phase]) return;
  cudaEvent_t e = prof_event(ctx);
  if (!e) return;
  cudaEventRecord(e, ctx->st);
  ctx->prof.pend[phase].push_back({ctx->prof.open[phase], e});
  ctx->prof.open[phase] = nullptr;
}

static void prof_collect(hci_ctx* ctx) {
  cudaStreamSynchronize(ctx->st);
  for (int k = 0; k < HCI_PH_COUNT; ++k) {
    for (auto& pr : ctx->prof.pend[k]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pr[0], pr[1]) == cudaSuccess) {
        ctx->prof.ms[k] += ms;
        ctx->prof.count[k] += 1;
      }
      ctx->prof.pool.push_back(pr[0]);
      ctx->prof.pool.push_back(pr[1]);
    }
    ctx->prof.pend[k].clear();
  }
}

void prof_release(hci_ctx* ctx) {
  prof_collect(ctx);
  for (int k = 0; k < HCI_PH_COUNT; ++k)
    if (ctx->prof.open[k]) { ctx->prof.pool.push_back(ctx->prof.open[k]); ctx->prof.open[k] = nullptr; }
  for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
  ctx->prof.pool.clear();
}

extern "C" hci_status hci_profile(hci_ctx* ctx, int enable) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_profile: null context");
  ctx->prof.on = enable != 0;
  return HCI_OK;
}

extern "C" hci_status hci_timers(hci_ctx* ctx, double* ms, int64_t* counts, int nphase) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_timers: null context");
  if (nphase < 0 || nphase > HCI_PH_COUNT) return hci_fail(ctx, HCI_ERR_INVALID, "hci_timers: bad nphase");
  prof_collect(ctx);
  for (int k = 0; k < nphase; ++k) {
    if (ms) ms[k] = ctx->prof.ms[k];
    if (counts) counts[k] = ctx->prof.count[k];
  }
  for (int k = 0; k < HCI_PH_COUNT; ++k) { ctx->prof.ms[k] = 0.0; ctx->prof.count[k] = 0; }
  return HCI_OK;
}

extern "C" int64_t hci_launch_count(void) { return (int64_t)g_hci_launches.load(); }
