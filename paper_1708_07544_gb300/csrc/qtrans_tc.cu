// Quarter transform of the integral rotation on the tensor cores
// (Sec. III.A: the active-space integrals depend on kappa through
// U = exp(kappa); (pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd) is computed as
// four quarter transforms out[J][p] = sum_a in[a][J] M[a][p], J < n^3).
//
// Each quarter transform is a dense (n^3 x n) by (n x n) product in FP64.
// This part's FP64 pipe (2 DFMA per clock per SM) is narrow and its tensor
// cores take no FP64 operands, so the product is carried out exactly in
// integers on the bf16 tensor cores (tcgen05.mma, accumulators in tensor
// memory) and rounded once to FP64 (the splitting of Ozaki et al., "Error-
// free transformations of matrix multiplication by using fast routines of
// matrix multiplication and its applications", Numer. Algorithms 2012):
//
//  * every row J of the left operand (the n values in[a][J] that are summed)
//    and every column p of U is put in fixed point against its own largest
//    binary exponent E: v = sign * sum_{s=1..8} d_s 2^(-7 s) * 2^(E - 1022)
//    with integer digits 0 <= d_s < 128 (56 bits; the part below 2^-56 of
//    the largest entry is dropped);
//  * a digit is exactly a bf16, the product of two digits is below 2^14,
//    and a sum of such products over K <= 64 entries and up to 8 digit
//    pairs stays below 2^23, so the FP32 accumulation of the tensor cores is
//    exact; the digit pairs (s, t) of one level L = s + t accumulate into
//    one tensor-memory column block;
//  * levels 2..10 are kept (2..9 when n > 48, where 9 blocks of 64 columns
//    would not fit the 512 columns of tensor memory); the pairs of higher
//    levels weigh at most about 2^-63 (2^-56) of the largest term;
//  * the epilogue reads the level sums, combines them exactly in 128-bit
//    integers and rounds once to FP64 (round to nearest even), scaled by
//    2^(E_J + E_p); results below the FP64 normal range are returned as 0.
//
// The error against the exact sum is thus about 2^-55 of
// max_a |in[a][J]| * max_a |M[a][p]| (levels to 10), of the order of an
// FP64 dot product's rounding error.
//
// Layout: one CTA per SM (persistent), 128 threads; thread m owns row
// J0 + m of the current tile of 128 rows in the split and in the epilogue
// (the four warps read tensor-memory lanes 32w..32w+31, the rows of the
// M = 128 accumulator).  The digits sit in shared memory in the canonical
// K-major layout without swizzle (8 x 16-byte core matrices); U's digits
// are made once per CTA.  The output tile (128 x n doubles, contiguous in
// global memory) is staged in shared memory and written coalesced.
#include <cuda.h>

#include "hci_internal.cuh"

namespace {

constexpr int QTC_M = 128;        // rows (J) per tile = accumulator lanes
constexpr int QTC_S = 8;          // digits per operand entry
constexpr int QTC_TMEM_COLS = 512;
constexpr long QTC_WAIT_LIMIT = 1L << 20;   // mbarrier polls before giving up

// set when a CTA gave up waiting for its products (never expected); read
// and cleared by the host after the rotation's final synchronisation
__device__ int g_qtc_timeout;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: canonical K-major layout, no swizzle;
// lbo = byte distance of core matrices adjacent in K, sbo = in M (or N)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: bf16 A and B (K-major), FP32 D,
// M = 128, N = np
__host__ __device__ constexpr uint32_t mma_idesc(int np) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(np >> 3) << 17) | ((uint32_t)(QTC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor cores
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
  for (long i = 0; i < QTC_WAIT_LIMIT; ++i)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

// 32 lanes x 8 columns of 32 bits: thread t gets lane (base lane + t)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// byte offset of element (row, k) in a K-major no-swizzle operand of kg
// 8-element groups along K
__device__ __forceinline__ uint32_t core_off(int row, int kgrp, int kg) {
  return (uint32_t)(((row >> 3) * kg + kgrp) * 128 + (row & 7) * 16);
}

// bf16 bits of the integer 0 <= c < 128 with the given sign bit: the FP32
// value of c, made exactly with one FP32 subtraction, has at most 7
// significant bits, so its upper half is c in bf16
__device__ __forceinline__ uint32_t digit_bf16(uint32_t c, uint32_t sign16) {
  const float f = __uint_as_float(0x4B000000u | c) - 8388608.0f;
  return (__float_as_uint(f) >> 16) | sign16;
}

// fixed point of one FP64 entry against the exponent e of its row (or
// column): 56 bits, value = fx 2^(e - 1078); the sign in bit 15 of *sign16
__device__ __forceinline__ uint64_t to_fixed(double v, int e, uint32_t* sign16) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int ev = (int)((b >> 52) & 0x7FF);
  *sign16 = (uint32_t)(b >> 48) & 0x8000u;
  if (ev == 0) return 0;   // zero (subnormals count as zero)
  const uint64_t m = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 3;
  const int sh = e - ev;
  return sh < 57 ? (m >> sh) : 0ull;
}

__device__ __forceinline__ int biased_exp(double v) {
  return (int)(((uint64_t)__double_as_longlong(v) >> 52) & 0x7FF);
}

// eight bf16 digits of slice s (1-based) of eight consecutive entries
__device__ __forceinline__ uint4 pack_slice(const uint64_t (&fx)[8], const uint32_t (&sg)[8], int s) {
  const int sh = 56 - 7 * s;
  uint32_t h[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] = digit_bf16((uint32_t)(fx[i] >> sh) & 127u, sg[i]);
  return make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
}

// S 2^e2 rounded to the nearest FP64 (ties to even); 0 below the normal range
__device__ __forceinline__ double round_scaled(__int128 S, int e2) {
  if (S == 0) return 0.0;
  const unsigned long long sign = S < 0 ? 0x8000000000000000ull : 0ull;
  unsigned __int128 m = S < 0 ? (unsigned __int128)(-S) : (unsigned __int128)S;
  const unsigned long long mh = (unsigned long long)(m >> 64), ml = (unsigned long long)m;
  const int lz = mh ? __clzll((long long)mh) : 64 + __clzll((long long)ml);
  m <<= lz;   // leading one at bit 127
  const unsigned long long top = (unsigned long long)(m >> 64), rest = (unsigned long long)m;
  unsigned long long mant = top >> 11;   // 53 bits
  const unsigned long long rb = top & 0x7FFull;
  if (rb > 0x400ull || (rb == 0x400ull && (rest != 0ull || (mant & 1ull)))) ++mant;
  const int e = 127 - lz + e2;   // exponent of the leading one
  if (e < -1022) return __longlong_as_double((long long)sign);
  if (e > 1023) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sign | (((unsigned long long)(e + 1022) << 52) + mant)));
}

template <int NP>
struct QtcCfg {
  static constexpr int KP = NP;                         // padded n along K
  static constexpr int KG = KP / 8;                     // core matrices along K
  static constexpr int LV = NP <= 48 ? 9 : 8;           // levels kept: 2 .. LV + 1
  static constexpr int A_SLICE = QTC_M * KP * 2;        // bytes of one digit slice of a tile
  static constexpr int B_SLICE = NP * KP * 2;
  static constexpr int A_BYTES = QTC_S * A_SLICE;
  static constexpr int B_BYTES = QTC_S * B_SLICE;
  static constexpr int OFF_B = A_BYTES;
  static constexpr int OFF_COLEXP = OFF_B + B_BYTES;
  static constexpr int OFF_MBAR = OFF_COLEXP + 64 * 4;
  static constexpr int OFF_SLOT = OFF_MBAR + 8;
  static constexpr int BYTES = OFF_SLOT + 8;
  // one CTA per SM, so that each CTA's tensor-memory allocation is served at once
  static constexpr int SMEM = (BYTES + 1024 > 120 * 1024 ? BYTES + 1024 : 120 * 1024);
  static_assert(LV * NP <= QTC_TMEM_COLS, "level blocks exceed tensor memory");
  static_assert(QTC_M * (NP + 1) * 8 <= A_BYTES, "output staging exceeds the digit buffer");
};

template <int NP>
__global__ void __launch_bounds__(QTC_M, 1) k_qtrans_tc(int n, const double* __restrict__ in,
                                                       const double* __restrict__ M, double* __restrict__ out,
                                                       int64_t ntiles) {
  using C = QtcCfg<NP>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* As = sm;
  uint8_t* Bs = sm + C::OFF_B;
  int* colexp = reinterpret_cast<int*>(sm + C::OFF_COLEXP);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + C::OFF_MBAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + C::OFF_SLOT);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t N3 = (int64_t)n * n * n;
  const uint32_t mbar_a = smem_u32(mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(QTC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // digits of U: operand B row p = column p of M, K index a
  if (tid < NP) {
    const int p = tid;
    int e = 0;
    if (p < n)
      for (int a = 0; a < n; ++a) e = max(e, biased_exp(M[a * n + p]));
    colexp[p] = e;
#pragma unroll 1
    for (int g = 0; g < C::KG; ++g) {
      uint64_t fx[8];
      uint32_t sg[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int a = g * 8 + i;
        fx[i] = (p < n && a < n) ? to_fixed(M[a * n + p], e, &sg[i]) : 0ull;
        if (!(p < n && a < n)) sg[i] = 0;
      }
#pragma unroll
      for (int s = 1; s <= QTC_S; ++s)
        *reinterpret_cast<uint4*>(Bs + (s - 1) * C::B_SLICE + core_off(p, g, C::KG)) = pack_slice(fx, sg, s);
    }
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *slot;
  const uint32_t As_a = smem_u32(As), Bs_a = smem_u32(Bs);
  constexpr uint32_t idesc = mma_idesc(NP);
  bool failed = false;
  uint32_t phase = 0;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t J0 = tile * QTC_M;
    const int64_t J = J0 + tid;
    const bool valid = J < N3;
    // this thread's row: load, exponent, digits
    double v[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) v[a] = (valid && a < n) ? __ldg(in + (int64_t)a * N3 + J) : 0.0;
    int e = 0;
#pragma unroll
    for (int a = 0; a < NP; ++a) e = max(e, biased_exp(v[a]));
#pragma unroll
    for (int g = 0; g < C::KG; ++g) {
      uint64_t fx[8];
      uint32_t sg[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) fx[i] = to_fixed(v[g * 8 + i], e, &sg[i]);
#pragma unroll
      for (int s = 1; s <= QTC_S; ++s)
        *reinterpret_cast<uint4*>(As + (s - 1) * C::A_SLICE + core_off(tid, g, C::KG)) = pack_slice(fx, sg, s);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
#pragma unroll 1
      for (int li = 0; li < C::LV; ++li) {
        const int L = li + 2;
        int acc = 0;
        for (int s = (L - QTC_S > 1 ? L - QTC_S : 1); s <= (L - 1 < QTC_S ? L - 1 : QTC_S); ++s) {
          const int t = L - s;
#pragma unroll
          for (int kk = 0; kk < C::KP / 16; ++kk) {
            const uint64_t ad = smem_desc(As_a + (s - 1) * C::A_SLICE + kk * 256, 128, C::KG * 128);
            const uint64_t bd = smem_desc(Bs_a + (t - 1) * C::B_SLICE + kk * 256, 128, C::KG * 128);
            mma_bf16(tmem + (uint32_t)(li * NP), ad, bd, idesc, acc);
            acc = 1;
          }
        }
      }
      mma_commit(mbar_a);
    }
    bool ok = mbar_wait_bounded(mbar_a, phase);
    if (!ok) {
      atomicExch(&g_qtc_timeout, 1);
      mbar_wait_bounded(mbar_a, phase);   // let products still in flight finish
    }
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    fence_after_sync();
    // epilogue: the level sums of this row, combined exactly and rounded;
    // staged in the (now free) digit buffer as rows of n + 1 doubles
    double* stage = reinterpret_cast<double*>(As);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int cc = 0; cc < NP / 8; ++cc) {
      uint32_t r[C::LV][8];
#pragma unroll
      for (int li = 0; li < C::LV; ++li) tmem_ld8(lane_base + (uint32_t)(li * NP + cc * 8), r[li]);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int p = cc * 8 + j;
        if (p >= n) break;
        // levels split in two exact 64-bit Horner sums (each level sum is
        // an integer below 2^23 in magnitude)
        constexpr int NLO = C::LV < 5 ? C::LV : 5;
        long long hi = 0, lo = 0;
#pragma unroll
        for (int li = 0; li < C::LV - NLO; ++li) hi = hi * 128 + __float2int_rn(__uint_as_float(r[li][j]));
#pragma unroll
        for (int li = C::LV - NLO; li < C::LV; ++li) lo = lo * 128 + __float2int_rn(__uint_as_float(r[li][j]));
        const __int128 S = ((__int128)hi << (7 * NLO)) + (__int128)lo;
        const int e2 = e + colexp[p] - 2044 - 7 * (C::LV + 1);
        stage[tid * (n + 1) + p] = (e == 0 || colexp[p] == 0) ? 0.0 : round_scaled(S, e2);
      }
    }
    fence_before_sync();
    __syncthreads();
    // the tile's rows are contiguous in out: write them coalesced
    const int64_t rows = (N3 - J0) < QTC_M ? (N3 - J0) : QTC_M;
    const int cnt = (int)rows * n;
    for (int i = tid; i < cnt; i += QTC_M) {
      const int m = i / n, p = i - m * n;
      out[J0 * n + i] = stage[m * (n + 1) + p];
    }
    __syncthreads();
  }
  (void)failed;
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(QTC_TMEM_COLS) : "memory");
}

int g_qtc_nsm[HCI_MAXORB];   // SM count per device ordinal (0: not looked up)

template <int NP>
hci_status launch(cudaStream_t st, int n, const double* in, const double* M, double* out) {
  using C = QtcCfg<NP>;
  static bool attr_set[HCI_MAXORB] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= HCI_MAXORB) return HCI_ERR_CUDA;
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(k_qtrans_tc<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess)
      return HCI_ERR_CUDA;
    attr_set[dev] = true;
  }
  if (g_qtc_nsm[dev] == 0) {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
      return HCI_ERR_CUDA;
    g_qtc_nsm[dev] = nsm;
  }
  const int64_t N3 = (int64_t)n * n * n;
  const int64_t ntiles = (N3 + QTC_M - 1) / QTC_M;
  const int grid = (int)(ntiles < g_qtc_nsm[dev] ? ntiles : g_qtc_nsm[dev]);
  HCI_LAUNCH(k_qtrans_tc<NP>, grid, QTC_M, C::SMEM, st)(n, in, M, out, ntiles);
  return cudaGetLastError() == cudaSuccess ? HCI_OK : HCI_ERR_CUDA;
}

}  // namespace

hci_status qtrans_tc(cudaStream_t st, int n, const double* in, const double* M, double* out) {
  if (n < 1 || n > HCI_MAXORB) return HCI_ERR_INVALID;
  if (n <= 16) return launch<16>(st, n, in, M, out);
  if (n <= 32) return launch<32>(st, n, in, M, out);
  if (n <= 48) return launch<48>(st, n, in, M, out);
  return launch<64>(st, n, in, M, out);
}

hci_status qtrans_tc_check(cudaStream_t st) {
  int flag = 0;
  if (cudaMemcpyFromSymbolAsync(&flag, g_qtc_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return HCI_ERR_CUDA;
  if (flag) {
    static const int zero = 0;
    cudaMemcpyToSymbolAsync(g_qtc_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
    return HCI_ERR_CUDA;
  }
  return HCI_OK;
}
