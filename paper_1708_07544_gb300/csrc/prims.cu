// Device-wide primitives: exclusive scan, stable LSD radix sort of 128-bit
// determinant keys, content hash and sortedness check of key arrays.
#include "hci_internal.cuh"

namespace {

constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t btot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t inc = warp_incl_scan(v);
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < nw ? wsum[lane] : 0;
    int64_t wi = warp_incl_scan(w);
    if (lane < nw) wsum[lane] = wi - w;
    if (lane == nw - 1) btot = wi;
  }
  __syncthreads();
  int64_t res = inc - v + wsum[warp];
  if (total) *total = btot;
  __syncthreads();
  return res;
}

__global__ void k_scan_reduce(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ bsum) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t acc = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)k * SCAN_BLOCK + threadIdx.x;
    if (i < n) acc += in[i];
  }
  int64_t tot;
  block_excl_scan(acc, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: exclusive scan of m block sums in place, total to *total
__global__ void k_scan_sums(int64_t* bsum, int64_t m, int64_t* total) {
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < m; b += blockDim.x) {
    int64_t i = b + threadIdx.x;
    int64_t v = i < m ? bsum[i] : 0;
    int64_t tot;
    int64_t ex = block_excl_scan(v, &tot);
    if (i < m) bsum[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_final(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             const int64_t* __restrict__ bsum) {
  // each thread owns SCAN_ITEMS consecutive elements
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t acc = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : 0;
    acc += v[k];
  }
  int64_t tot;
  int64_t ex = block_excl_scan(acc, &tot) + bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
}

// ---------------------------------------------------------------------------
// radix sort of 128-bit keys, 8-bit digits, stable per pass
// ---------------------------------------------------------------------------
constexpr int RS_BLOCK = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_BLOCK * RS_ITEMS;

__device__ __forceinline__ int digit_of(ulonglong2 k, int word, int shift) {
  uint64_t w = word == 0 ? k.y : k.x;   // word 0 = low (beta) word, 1 = high (alpha)
  return (int)((w >> shift) & 0xFFu);
}

__global__ void k_rs_hist(const ulonglong2* __restrict__ keys, int64_t n, int word, int shift,
                          int64_t* __restrict__ hist, int64_t ntiles) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int k = 0; k < RS_ITEMS; ++k) {
    int64_t i = base + (int64_t)k * RS_BLOCK + threadIdx.x;
    if (i < n) atomicAdd(&h[digit_of(keys[i], word, shift)], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const ulonglong2* __restrict__ in, ulonglong2* __restrict__ out, int64_t n,
                             int word, int shift, const int64_t* __restrict__ offs, int64_t ntiles,
                             const double* __restrict__ pin, double* __restrict__ pout,
                             const int32_t* __restrict__ qin, int32_t* __restrict__ qout) {
  __shared__ int64_t base[256];
  __shared__ int wcnt[RS_BLOCK / 32][256];
  __shared__ int tot[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ITEMS; ++r) {
    int64_t i = (int64_t)blockIdx.x * RS_TILE + (int64_t)r * RS_BLOCK + tid;
    bool valid = i < n;
    ulonglong2 key = valid ? in[i] : make_ulonglong2(0, 0);
    int d = valid ? digit_of(key, word, shift) : 256;
    for (int k = tid; k < (RS_BLOCK / 32) * 256; k += RS_BLOCK) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & lt);
    int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      int run = 0;
      for (int w = 0; w < RS_BLOCK / 32; ++w) {
        int c = wcnt[w][tid];
        wcnt[w][tid] = run;
        run += c;
      }
      tot[tid] = run;
    }
    __syncthreads();
    if (valid) {
      const int64_t dst = base[d] + wcnt[warp][d] + rank;
      out[dst] = key;
      if (pin) pout[dst] = pin[i];
      if (qin) qout[dst] = qin[i];
    }
    __syncthreads();
    base[tid] += tot[tid];
    __syncthreads();
  }
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33;
  return x;
}

__global__ void k_hash(const ulonglong2* __restrict__ keys, int64_t n, unsigned long long* out) {
  uint64_t hx = 0, hs = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 k = keys[i];
    uint64_t m = mix64(k.x * 0x9E3779B97F4A7C15ull ^ mix64(k.y + (uint64_t)i));
    hx ^= m;
    hs += m;
  }
  for (int o = 16; o; o >>= 1) {
    hx ^= __shfl_xor_sync(0xffffffffu, hx, o);
    hs += __shfl_xor_sync(0xffffffffu, hs, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicXor(&out[0], (unsigned long long)hx);
    atomicAdd(&out[1], (unsigned long long)hs);
  }
}

__global__ void k_check_sorted(const ulonglong2* __restrict__ keys, int64_t n, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < n; i += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 a = keys[i], b = keys[i + 1];
    bool ok = (a.x < b.x) || (a.x == b.x && a.y < b.y);
    if (!ok) atomicOr(bad, 1);
  }
}

}  // namespace

hci_status scan_i64(hci_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev) {
  if (n <= 0) {
    if (total_dev) HCI_CUDA(ctx, cudaMemsetAsync(total_dev, 0, sizeof(int64_t), ctx->st));
    return HCI_OK;
  }
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  HCI_TRY(ensure_buf(ctx, ctx->s_scan, (size_t)nb * sizeof(int64_t)));
  int64_t* bsum = bp<int64_t>(ctx->s_scan);
  HCI_LAUNCH(k_scan_reduce, (unsigned)nb, SCAN_BLOCK, 0, ctx->st)(in, n, bsum);
  HCI_LAUNCH(k_scan_sums, 1, 1024, 0, ctx->st)(bsum, nb, total_dev);
  HCI_LAUNCH(k_scan_final, (unsigned)nb, SCAN_BLOCK, 0, ctx->st)(in, out, n, bsum);
  HCI_CUDA(ctx, cudaGetLastError());
  return HCI_OK;
}

hci_status sort_keys(hci_ctx* ctx, uint64_t* keys, uint64_t* tmp, int64_t n, int bits_a, int bits_b) {
  return sort_pairs(ctx, keys, tmp, nullptr, nullptr, nullptr, nullptr, n, bits_a, bits_b);
}

hci_status sort_pairs(hci_ctx* ctx, uint64_t* keys, uint64_t* tmp, double* vals, double* vtmp, int32_t* idx,
                      int32_t* itmp, int64_t n, int bits_a, int bits_b) {
  if (n <= 1) return HCI_OK;
  int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  HCI_TRY(ensure_buf(ctx, ctx->s_hist, (size_t)ntiles * 256 * 2 * sizeof(int64_t)));
  int64_t* hist = bp<int64_t>(ctx->s_hist);
  int64_t* offs = hist + ntiles * 256;
  ulonglong2* a = reinterpret_cast<ulonglong2*>(keys);
  ulonglong2* b = reinterpret_cast<ulonglong2*>(tmp);
  double* va = vals;
  double* vb = vtmp;
  int32_t* ia = idx;
  int32_t* ib = itmp;
  int passes = 0;
  for (int word = 0; word < 2; ++word) {
    int bits = word == 0 ? bits_b : bits_a;
    for (int shift = 0; shift < bits; shift += 8) {
      HCI_LAUNCH(k_rs_hist, (unsigned)ntiles, RS_BLOCK, 0, ctx->st)(a, n, word, shift, hist, ntiles);
      HCI_TRY(scan_i64(ctx, hist, offs, ntiles * 256, nullptr));
      HCI_LAUNCH(k_rs_scatter, (unsigned)ntiles, RS_BLOCK, 0, ctx->st)(a, b, n, word, shift, offs, ntiles, va, vb,
                                                                       ia, ib);
      ulonglong2* t = a; a = b; b = t;
      double* tv = va; va = vb; vb = tv;
      int32_t* ti = ia; ia = ib; ib = ti;
      ++passes;
    }
  }
  HCI_CUDA(ctx, cudaGetLastError());
  if (passes & 1) {
    HCI_CUDA(ctx, cudaMemcpyAsync(keys, tmp, (size_t)n * 16, cudaMemcpyDeviceToDevice, ctx->st));
    if (vals) HCI_CUDA(ctx, cudaMemcpyAsync(vals, vtmp, (size_t)n * 8, cudaMemcpyDeviceToDevice, ctx->st));
    if (idx) HCI_CUDA(ctx, cudaMemcpyAsync(idx, itmp, (size_t)n * 4, cudaMemcpyDeviceToDevice, ctx->st));
  }
  return HCI_OK;
}

hci_status hash_keys(hci_ctx* ctx, const uint64_t* keys, int64_t n, uint64_t* hash_host) {
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  unsigned long long* d = bp<unsigned long long>(ctx->s_counter);
  HCI_CUDA(ctx, cudaMemsetAsync(d, 0, 16, ctx->st));
  if (n > 0)
    HCI_LAUNCH(k_hash, grid_for(n, 256, ctx->nsm * 8), 256, 0, ctx->st)(reinterpret_cast<const ulonglong2*>(keys), n, d);
  unsigned long long hv[2];
  HCI_CUDA(ctx, cudaMemcpyAsync(hv, d, 16, cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  *hash_host = (uint64_t)hv[0] * 31ull + (uint64_t)hv[1] + (uint64_t)n * 0x9E3779B97F4A7C15ull;
  return HCI_OK;
}

hci_status check_sorted(hci_ctx* ctx, const uint64_t* keys, int64_t n, int* ok_host) {
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  int* d = reinterpret_cast<int*>(bp<char>(ctx->s_counter) + 32);
  HCI_CUDA(ctx, cudaMemsetAsync(d, 0, sizeof(int), ctx->st));
  if (n > 1)
    HCI_LAUNCH(k_check_sorted, grid_for(n, 256, ctx->nsm * 8), 256, 0, ctx->st)(reinterpret_cast<const ulonglong2*>(keys), n, d);
  int bad = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&bad, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  *ok_host = bad ? 0 : 1;
  return HCI_OK;
}
