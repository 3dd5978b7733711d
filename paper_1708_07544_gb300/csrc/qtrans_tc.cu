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
//    binary exponent E: x = v 2^(1077 - E), a signed integer |x| < 2^55
//    (the part below 2^-55 of the largest entry is dropped), written in
//    seven balanced base-256 digits, x = sum_{s=1..7} d_s 256^(7-s) with
//    -128 <= d_s <= 127 (the bytes of x + 0x80808080808080, less 128;
//    the leading digit takes the carry into bit 56 and reaches 128);
//  * a digit is exactly a bf16, the product of two digits is at most 2^14
//    in magnitude, and a sum of such products over K <= 64 entries and up
//    to 7 digit pairs stays below 2^23, so the FP32 accumulation of the
//    tensor cores is exact; the digit pairs (s, t) of one level L = s + t
//    accumulate into one block of n (rounded up to 16) tensor-memory
//    columns;
//  * levels 2..9 are kept (8 blocks, at most 512 columns); the pairs of
//    the higher levels weigh at most about 2^-64 of the largest term;
//  * the epilogue reads the level sums, combines them exactly in 64-bit
//    integers (an 80-bit sum in two words) and rounds once to FP64 (to
//    nearest, ties to even), scaled by 2^(E_J + E_p); results below the
//    FP64 normal range are returned as 0.
//
// The error against the exact sum is thus about 2^-55 n of
// max_a |in[a][J]| * max_a |M[a][p]| at worst (the digit truncation), of
// the order of an FP64 dot product's rounding error, but normwise: an
// entry far below the rest of its row keeps an absolute error of that size
// where an FP64 dot product's error is componentwise.
//
// Layout: one CTA per SM (persistent), 16 warps.  In the split four
// threads share a row of the current tile of 128 rows (each takes every
// fourth group of 8 entries; the row's exponent is the maximum of their
// partial maxima), and each thread's entries of the next tile are loaded
// while the tensor cores work on this one; in the epilogue warp w reads
// tensor-memory lanes 32 (w mod 4) .. + 31 (the rows of the M = 128
// accumulator) and every fourth group of 4 columns.  The digits sit in
// shared memory in the canonical K-major layout without swizzle (8 x
// 16-byte core matrices); U's digits are made once per CTA.  The output tile (128 x n doubles, contiguous in
// global memory) is staged in shared memory and written coalesced.
#include <cuda.h>

#include "hci_internal.cuh"

namespace {

constexpr int QTC_M = 128;        // rows (J) per tile = accumulator lanes
constexpr int QTC_S = 7;          // balanced base-256 digits per operand entry
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

// 32 lanes x 4 columns of 32 bits: thread t gets lane (base lane + t)
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// byte offset of element (row, k) in a K-major no-swizzle operand of kg
// 8-element groups along K
__device__ __forceinline__ uint32_t core_off(int row, int kgrp, int kg) {
  return (uint32_t)(((row >> 3) * kg + kgrp) * 128 + (row & 7) * 16);
}

__device__ __forceinline__ int biased_exp(double v) {
  return (int)(((uint64_t)__double_as_longlong(v) >> 52) & 0x7FF);
}

// fixed point of one FP64 entry against the exponent e of its row (or
// column), x = v 2^(1077 - e) truncated (|x| < 2^55), returned as
// x + 0x80808080808080: its bytes 5..0 and its bits 48 and up, less 128,
// are the balanced digits d_7..d_2 and d_1 of x
constexpr uint64_t QTC_BIAS = 0x0080808080808080ull;
__device__ __forceinline__ uint64_t to_digits(double v, int e) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int ev = (int)((b >> 52) & 0x7FF);
  if (ev == 0) return QTC_BIAS;   // zero (subnormals count as zero)
  const uint64_t m = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 2;
  const int sh = e - ev;
  const uint64_t x = sh < 56 ? (m >> sh) : 0ull;
  return ((int64_t)b < 0 ? QTC_BIAS - x : QTC_BIAS + x);
}

// bf16 of digit s (1-based) of eight consecutive entries, packed in pairs:
// the byte b of y placed under the FP32 exponent of 2^23 gives 2^23 + b,
// less 2^23 + 128 the digit, exactly, with at most 8 significant bits, so
// the upper half of the FP32 value is the digit in bf16.  The leading digit
// takes all of y >> 48 (0 .. 256): x up to 2^55 - 1 carries into bit 56,
// so d_1 ranges over -128 .. 128, still exact in bf16 and still at most
// 2^14 in any digit product.
__device__ __forceinline__ uint4 pack_slice(const uint64_t (&y)[8], int s) {
  const int byte = 7 - s;                       // 6 .. 0
  const unsigned sel = (7u << 12) | (5u << 8) | (4u << 4) | (unsigned)(byte & 3);
  uint32_t f[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t w = byte >= 4 ? (uint32_t)(y[i] >> 32) : (uint32_t)y[i];
    const uint32_t bits = s == 1 ? (0x4B000000u | (uint32_t)(y[i] >> 48)) : __byte_perm(w, 0x4B000000u, sel);
    f[i] = __float_as_uint(__uint_as_float(bits) - 8388736.0f);
  }
  return make_uint4(__byte_perm(f[0], f[1], 0x7632), __byte_perm(f[2], f[3], 0x7632),
                    __byte_perm(f[4], f[5], 0x7632), __byte_perm(f[6], f[7], 0x7632));
}

// (T 2^32 + b) 2^e2 rounded to the nearest FP64 (ties to even), for
// |T| < 2^47 and 0 <= b < 2^32; 0 below the normal range.  The magnitude
// (at most 79 bits) is normalised into one 64-bit word: exactly when it is
// below 2^63, else its top 64 bits with the rest of b as sticky bits.
__device__ __forceinline__ double round_tb(long long T, uint32_t b, int e2) {
  if (T == 0 && b == 0u) return 0.0;
  const unsigned long long sign = T < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long Tm = T < 0 ? (unsigned long long)(-T) - (b != 0u ? 1ull : 0ull) : (unsigned long long)T;
  const uint32_t bm = T < 0 ? 0u - b : b;
  unsigned long long X;
  int e;
  bool sticky;
  if ((Tm >> 31) == 0ull) {
    const unsigned long long Y = (Tm << 32) | bm;
    const int lz = __clzll((long long)Y);
    X = Y << lz;
    e = 63 - lz + e2;
    sticky = false;
  } else {
    const int lz = __clzll((long long)Tm);   // 17 .. 32
    X = (Tm << lz) | (unsigned long long)(bm >> (32 - lz));
    sticky = (bm & ((1u << (32 - lz)) - 1u)) != 0u;
    e = 95 - lz + e2;
  }
  unsigned long long mant = X >> 11;   // 53 bits
  const unsigned long long rb = X & 0x7FFull;
  if (rb > 0x400ull || (rb == 0x400ull && (sticky || (mant & 1ull)))) ++mant;
  if (e < -1022) return __longlong_as_double((long long)sign);
  if (e > 1023) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sign | (((unsigned long long)(e + 1022) << 52) + mant)));
}

template <int NP>
struct QtcCfg {
  static constexpr int KP = NP;                         // padded n along K
  static constexpr int KG = KP / 8;                     // core matrices along K
  static constexpr int LV = 8;                          // levels kept: 2 .. 9
  // threads per row in the split and warps per lane group in the epilogue
  // (three, which shares the 6 entry groups and 12 column groups of
  // n <= 48 evenly, measured slower: fewer warps hide less latency)
  static constexpr int PARTS = 4;
  static constexpr int THREADS = QTC_M * PARTS;
  static constexpr int CS = 256 / NP < QTC_S ? 256 / NP : QTC_S;   // digit slices of U per MMA (N <= 256)
  static constexpr int A_SLICE = QTC_M * KP * 2;        // bytes of one digit slice of a tile
  static constexpr int B_SLICE = NP * KP * 2;
  static constexpr int A_BYTES = QTC_S * A_SLICE;
  static constexpr int B_BYTES = QTC_S * B_SLICE;
  static constexpr int OFF_B = A_BYTES;
  static constexpr int OFF_ROWEXP = OFF_B + B_BYTES;    // 4 partial maxima per row
  static constexpr int OFF_COLEXP = OFF_ROWEXP + 4 * QTC_M * 4;
  static constexpr int OFF_MBAR = OFF_COLEXP + 64 * 4;
  static constexpr int OFF_SLOT = OFF_MBAR + 8;
  static constexpr int BYTES = OFF_SLOT + 8;
  // one CTA per SM, so that each CTA's tensor-memory allocation is served at once
  static constexpr int SMEM = (BYTES + 1024 > 120 * 1024 ? BYTES + 1024 : 120 * 1024);
  static_assert(LV * NP <= QTC_TMEM_COLS, "level blocks exceed tensor memory");
  static_assert(LV == 8, "the epilogue combines levels 2..9");
  static_assert(QTC_M * (NP + 1) * 8 <= A_BYTES, "output staging exceeds the digit buffer");
};

// One tile's digit products (issued by one thread).  Digit pair (s, t)
// adds into the block of level s + t; U's digit slices lie one after the
// other along N with the same stride as its 8-row groups, so one MMA takes
// CS consecutive slices t0 .. t0 + CS - 1 of U against slice s of the tile
// and writes CS consecutive level blocks.  The first MMA into each block
// overwrites it: slice s = 1 reaches levels 2 .. 8, level 9 is first
// reached by (s, t) = (2, 7).
template <int NP>
__device__ __forceinline__ void issue_products(uint32_t tmem, uint32_t As_a, uint32_t Bs_a) {
  using C = QtcCfg<NP>;
  constexpr uint32_t SBO = C::KG * 128;
  auto issue = [&](int s, int t0, int cnt, bool acc0) {
#pragma unroll
    for (int kk = 0; kk < C::KP / 16; ++kk) {
      const uint64_t ad = smem_desc(As_a + (s - 1) * C::A_SLICE + kk * 256, 128, SBO);
      const uint64_t bd = smem_desc(Bs_a + (t0 - 1) * C::B_SLICE + kk * 256, 128, SBO);
      mma_bf16(tmem + (uint32_t)((s + t0 - 2) * NP), ad, bd, mma_idesc(cnt * NP), (kk > 0 || acc0) ? 1 : 0);
    }
  };
#pragma unroll 1
  for (int s = 1; s <= QTC_S; ++s) {
    int tmax = C::LV + 1 - s < QTC_S ? C::LV + 1 - s : QTC_S;
    if (s == 2) {
      issue(2, QTC_S, 1, false);
      tmax = QTC_S - 1;
    }
    for (int t0 = 1; t0 <= tmax; t0 += C::CS) issue(s, t0, tmax - t0 + 1 < C::CS ? tmax - t0 + 1 : C::CS, s > 1);
  }
}

template <int NP>
__global__ void __launch_bounds__(QtcCfg<NP>::THREADS, 1) k_qtrans_tc(int n, const double* __restrict__ in,
                                                             const double* __restrict__ M, double* __restrict__ out,
                                                             int64_t ntiles) {
  using C = QtcCfg<NP>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* As = sm;
  uint8_t* Bs = sm + C::OFF_B;
  int* rowexp = reinterpret_cast<int*>(sm + C::OFF_ROWEXP);
  int* colexp = reinterpret_cast<int*>(sm + C::OFF_COLEXP);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + C::OFF_MBAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + C::OFF_SLOT);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
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
      uint64_t y[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int a = g * 8 + i;
        y[i] = (p < n && a < n) ? to_digits(M[a * n + p], e) : QTC_BIAS;
      }
#pragma unroll
      for (int s = 1; s <= QTC_S; ++s)
        *reinterpret_cast<uint4*>(Bs + (s - 1) * C::B_SLICE + core_off(p, g, C::KG)) = pack_slice(y, s);
    }
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *slot;
  const uint32_t As_a = smem_u32(As), Bs_a = smem_u32(Bs);
  uint32_t phase = 0;
  // split: thread (row m, part q) takes the K groups q, q + 4, ... of row m
  const int m_split = tid & (QTC_M - 1), q_split = tid >> 7;
  // epilogue: warp w reads accumulator lanes 32 (w & 3) .. + 31 (its rows)
  // and the column groups (w >> 2), (w >> 2) + 4, ...
  const int m_epi = ((warp & 3) << 5) + lane, q_epi = warp >> 2;
  constexpr int GPT = (C::KG + C::PARTS - 1) / C::PARTS;   // K groups per thread at most

  // this thread's entries of a tile: K groups q_split, q_split + 4, ...
  // of row m_split, loaded one tile ahead so that the loads of the next
  // tile are in flight during this tile's products and epilogue
  double v[GPT][8];
  auto load_tile = [&](int64_t tile) {
    const int64_t J = tile * QTC_M + m_split;
    const bool valid = tile < ntiles && J < N3;
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      const int g = q_split + j * C::PARTS;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int a = g * 8 + i;
        v[j][i] = (g < C::KG && valid && a < n) ? __ldg(in + (int64_t)a * N3 + J) : 0.0;
      }
    }
  };
  load_tile(blockIdx.x);

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t J0 = tile * QTC_M;
    {
      int e = 0;
#pragma unroll
      for (int j = 0; j < GPT; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) e = max(e, biased_exp(v[j][i]));
      rowexp[q_split * QTC_M + m_split] = e;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < C::PARTS; ++q) e = max(e, rowexp[q * QTC_M + m_split]);
#pragma unroll
      for (int j = 0; j < GPT; ++j) {
        const int g = q_split + j * C::PARTS;
        if (g >= C::KG) break;
        uint64_t y[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) y[i] = to_digits(v[j][i], e);
#pragma unroll
        for (int s = 1; s <= QTC_S; ++s)
          *reinterpret_cast<uint4*>(As + (s - 1) * C::A_SLICE + core_off(m_split, g, C::KG)) = pack_slice(y, s);
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      issue_products<NP>(tmem, As_a, Bs_a);
      mma_commit(mbar_a);
    }
    load_tile(tile + gridDim.x);
    // one warp polls the barrier; the others wait at the block barrier
    bool ok = true;
    if (warp == 0) {
      ok = mbar_wait_bounded(mbar_a, phase);
      if (!ok) {
        atomicExch(&g_qtc_timeout, 1);
        mbar_wait_bounded(mbar_a, phase);   // let products still in flight finish
      }
    }
    phase ^= 1u;
    if (__syncthreads_or(!ok)) break;
    fence_after_sync();
    // epilogue: the level sums of this row, combined exactly and rounded;
    // staged in the (now free) digit buffer as rows of n + 1 doubles
    {
      double* stage = reinterpret_cast<double*>(As);
      int e = 0;
#pragma unroll
      for (int q = 0; q < C::PARTS; ++q) e = max(e, rowexp[q * QTC_M + m_epi]);
      const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
      for (int cc = q_epi; cc < NP / 4; cc += C::PARTS) {
        uint32_t r[C::LV][4];
#pragma unroll
        for (int li = 0; li < C::LV; ++li) tmem_ld4(lane_base + (uint32_t)(li * NP + cc * 4), r[li]);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int p = cc * 4 + j;
          if (p >= n) break;
          // S = sum_L D_L 256^(9 - L) (each level sum D_L an integer below
          // 2^23 in magnitude): pairs of levels in 32 bits, then levels
          // 2..5 and 6..9 in 64 bits, S = hi 2^32 + lo = T 2^32 + b; the
          // product is S 2^(E_J + E_p - 2114)
          int d[8];
#pragma unroll
          for (int li = 0; li < 8; ++li) d[li] = __float2int_rn(__uint_as_float(r[li][j]));
          const long long hi = (long long)(d[0] * 256 + d[1]) * 65536 + (d[2] * 256 + d[3]);
          const long long lo = (long long)(d[4] * 256 + d[5]) * 65536 + (d[6] * 256 + d[7]);
          const long long T = hi + (lo >> 32);
          const int ce = colexp[p];
          const int e2 = e + ce - 2114;
          stage[m_epi * (n + 1) + p] = (e == 0 || ce == 0) ? 0.0 : round_tb(T, (uint32_t)lo, e2);
        }
      }
    }
    fence_before_sync();
    __syncthreads();
    // the tile's rows are contiguous in out: write them coalesced
    {
      const double* stage = reinterpret_cast<const double*>(As);
      const int64_t rows = (N3 - J0) < QTC_M ? (N3 - J0) : QTC_M;
      const int cnt = (int)rows * n;
      // i / n as (i ceil(2^20 / n)) >> 20, exact for i < 2^13, n <= 64
      const uint32_t inv = ((1u << 20) + (uint32_t)n - 1u) / (uint32_t)n;
      for (int i = tid; i < cnt; i += C::THREADS) {
        const int m = (int)(((uint32_t)i * inv) >> 20), p = i - m * n;
        out[J0 * n + i] = stage[m * (n + 1) + p];
      }
    }
    __syncthreads();
  }
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
  HCI_LAUNCH(k_qtrans_tc<NP>, grid, C::THREADS, C::SMEM, st)(n, in, M, out, ntiles);
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
