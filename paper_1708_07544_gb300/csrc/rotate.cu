// Active-active orbital rotation of the integrals and its adjoint
// (Sec. III.A: the integrals depend on kappa through U = exp(kappa);
// Sec. III.B, Eq. vdedk2: dE/dkappa = sum dH/dkappa contracted with the RDMs).
//
// Forward:  h' = U^T h U,  (pq|rs)' = sum U_ap U_bq U_cr U_ds (ab|cd)
//           as four quarter transforms out[J][p] = sum_a in[a][J] M[a][p]
//           that each rotate the leading index to the back.
// Backward: dE/dh = U g1 U^T, dE/d(ab|cd) = sum D_pqrs U_ap U_bq U_cr U_ds
//           with D = rdm2/2, and dE/dU = h U g1^T + h^T U g1 + 4 sum_bcd
//           (xb|cd) T[y][b][c][d], T = D with its last three indices
//           back-transformed (the four index positions of a real state with
//           8-fold symmetric integrals contribute equally);
//           dE/dkappa = L_exp(kappa^T, dE/dU), the Frechet derivative of
//           exp at kappa^T, read off exp([[k^T, G], [0, k^T]]).
// The quarter transforms (the n^5 part) run on the bf16 tensor cores as
// exact digit products rounded once to FP64 (qtrans_tc.cu); the n x n
// matrix work stays on the FP64 pipe.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "hci_internal.cuh"

namespace {

// C = alpha * op(A) op(B) + beta * C, m x m row-major, one thread per entry
__global__ void k_mm(int m, const double* __restrict__ A, int tA, const double* __restrict__ B, int tB,
                     double* __restrict__ C, double alpha, double beta) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * m) return;
  int i = t / m, j = t % m;
  double acc = 0.0;
  for (int k = 0; k < m; ++k) {
    double a = tA ? A[k * m + i] : A[i * m + k];
    double b = tB ? B[j * m + k] : B[k * m + j];
    acc = fma(a, b, acc);
  }
  C[t] = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * C[t]);
}

// E = I + X * E / k   (Horner step of the Taylor series), X E in tmp
__global__ void k_horner(int m, const double* __restrict__ XE, double* __restrict__ E, double invk) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * m) return;
  int i = t / m, j = t % m;
  E[t] = (i == j ? 1.0 : 0.0) + XE[t] * invk;
}

__global__ void k_eye_plus(int m, const double* __restrict__ X, double s, double* __restrict__ E) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * m) return;
  int i = t / m, j = t % m;
  E[t] = (i == j ? 1.0 : 0.0) + s * X[t];
}

__global__ void k_scale_copy(int64_t cnt, const double* __restrict__ in, double s, double* __restrict__ out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = s * in[t];
}

// max column abs-sum (1-norm) of an m x m matrix, single block
__global__ void k_norm1(int m, const double* __restrict__ A, double* out) {
  __shared__ double s[1024];
  double v = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double cs = 0.0;
    for (int i = 0; i < m; ++i) cs += fabs(A[i * m + j]);
    v = fmax(v, cs);
  }
  s[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) r = fmax(r, s[t]);
    *out = r;
  }
}

// block matrix [[K^T, G], [0, K^T]] of size 2n
__global__ void k_frechet_block(int n, const double* __restrict__ K, const double* __restrict__ G, double* __restrict__ B) {
  int m = 2 * n;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * m) return;
  int i = t / m, j = t % m;
  double v = 0.0;
  if (i < n && j < n) v = K[j * n + i];
  else if (i >= n && j >= n) v = K[(j - n) * n + (i - n)];
  else if (i < n && j >= n) v = G[i * n + (j - n)];
  B[t] = v;
}

__global__ void k_upper_right(int n, const double* __restrict__ B, double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  int i = t / n, j = t % n;
  out[t] = B[i * 2 * n + n + j];
}

__global__ void k_eye(int n, double* __restrict__ I) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n * n) I[t] = (t / n == t % n) ? 1.0 : 0.0;
}

// The solver reads different permutations of one integral (heat-bath lists,
// Slater-Condon rules), so every permutation must hold the same bits: each
// element of the 8-fold orbit of (pq|rs) takes the value of the orbit's
// representative ((a,b) = sorted (p,q), (c,d) = sorted (r,s), pairs ordered
// so that (a,b) <= (c,d)), and h_pq = h_qp takes the value of h_min,max.  In
// place: a representative is only ever rewritten with its own value.
__global__ void k_sym8(int n, double* __restrict__ eri) {
  const int64_t n2 = (int64_t)n * n, n4 = n2 * n2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t % n), r = (int)((t / n) % n), q = (int)((t / n2) % n), p = (int)(t / (n2 * n));
    int a = p < q ? p : q, b = p < q ? q : p, c = r < s ? r : s, d = r < s ? s : r;
    if (a * n + b > c * n + d) {
      const int ta = a, tb = b;
      a = c; b = d; c = ta; d = tb;
    }
    const int64_t rep = (((int64_t)a * n + b) * n + c) * n + d;
    if (rep != t) eri[t] = eri[rep];
  }
}
__global__ void k_symh(int n, double* __restrict__ h) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int p = t / n, q = t % n;
  if (p > q) h[t] = h[q * n + p];
}

// partial[b][x][y] = sum_{J in chunk b} A[x][J] B[y][J]  (A, B: n x K)
constexpr int NT_CH = 64;
__global__ void __launch_bounds__(256) k_gemm_nt_part(int n, int64_t K, const double* __restrict__ A,
                                                      const double* __restrict__ B, double* __restrict__ partial) {
  extern __shared__ double sm[];
  double* At = sm;                 // n * NT_CH
  double* Bt = sm + n * NT_CH;     // n * NT_CH
  const int64_t J0 = (int64_t)blockIdx.x * NT_CH;
  for (int t = threadIdx.x; t < n * NT_CH; t += blockDim.x) {
    int x = t / NT_CH, jj = t % NT_CH;
    int64_t J = J0 + jj;
    At[t] = J < K ? A[(int64_t)x * K + J] : 0.0;
    Bt[t] = J < K ? B[(int64_t)x * K + J] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int x = t / n, y = t % n;
    double acc = 0.0;
    for (int jj = 0; jj < NT_CH; ++jj) acc = fma(At[x * NT_CH + jj], Bt[y * NT_CH + jj], acc);
    partial[(int64_t)blockIdx.x * n * n + t] = acc;
  }
}

__global__ void k_sum_parts(int nn, int nparts, const double* __restrict__ partial, double scale,
                            double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nn) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += partial[(int64_t)b * nn + t];
  out[t] += scale * s;
}

struct Scratch {
  cudaStream_t st;
  void* ptrs[16];
  int count = 0;
  int64_t left = hci_fail_alloc_env();   // host-side fault injection (tests)
  double* get(size_t doubles) {
    void* p = nullptr;
    if (left == 0) return nullptr;
    if (left > 0) --left;
    if (cudaMallocAsync(&p, doubles * 8 + 64, st) != cudaSuccess) return nullptr;
    ptrs[count++] = p;
    return reinterpret_cast<double*>(p);
  }
  ~Scratch() {
    for (int i = 0; i < count; ++i) cudaFreeAsync(ptrs[i], st);
  }
};

inline unsigned blocks(int64_t work, int b = 256) { return (unsigned)((work + b - 1) / b); }

hci_status mm(cudaStream_t st, int m, const double* A, int tA, const double* B, int tB, double* C, double alpha,
              double beta) {
  HCI_LAUNCH(k_mm, blocks((int64_t)m * m), 256, 0, st)(m, A, tA, B, tB, C, alpha, beta);
  return HCI_OK;
}

// E = exp(A) for an m x m matrix; w1, w2, w3 scratch of m*m
hci_status expm_dev(cudaStream_t st, int m, const double* A, double* E, double* w1, double* w2, double* w3,
                    double* dscal) {
  HCI_LAUNCH(k_norm1, 1, 256, 0, st)(m, A, dscal);
  double nrm = 0.0;
  if (cudaMemcpyAsync(&nrm, dscal, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HCI_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HCI_ERR_CUDA;
  if (!std::isfinite(nrm)) return HCI_ERR_INVALID;
  int s = 0;
  while (nrm / std::ldexp(1.0, s) > 0.5) ++s;
  const double sc = std::ldexp(1.0, -s);
  HCI_LAUNCH(k_scale_copy, blocks((int64_t)m * m), 256, 0, st)((int64_t)m * m, A, sc, w1);   // X
  // Horner: E = I + X/18; E = I + X E / k for k = 17..1
  const int deg = 18;
  HCI_LAUNCH(k_eye_plus, blocks((int64_t)m * m), 256, 0, st)(m, w1, 1.0 / deg, E);
  for (int k = deg - 1; k >= 1; --k) {
    mm(st, m, w1, 0, E, 0, w2, 1.0, 0.0);
    HCI_LAUNCH(k_horner, blocks((int64_t)m * m), 256, 0, st)(m, w2, E, 1.0 / k);
  }
  for (int i = 0; i < s; ++i) {
    mm(st, m, E, 0, E, 0, w3, 1.0, 0.0);
    cudaMemcpyAsync(E, w3, (size_t)m * m * 8, cudaMemcpyDeviceToDevice, st);
  }
  return cudaGetLastError() == cudaSuccess ? HCI_OK : HCI_ERR_CUDA;
}

// out[J*n + p] = sum_a in[a*N3 + J] * M[a*n + p], J < N3 = n^3
#define QTRANS(who, in, M, out)                                                              \
  do {                                                                                       \
    if (qtrans_tc(st, n, in, M, out) != HCI_OK)                                              \
      return hci_fail(nullptr, HCI_ERR_CUDA, who ": quarter transform launch failed: %s",     \
                      cudaGetErrorString(cudaGetLastError()));                               \
  } while (0)

// after the final synchronisation: the quarter transforms completed
#define QTRANS_CHECK(who)                                                                        \
  do {                                                                                           \
    if (qtrans_tc_check(st) != HCI_OK)                                                             \
      return hci_fail(nullptr, HCI_ERR_CUDA, who ": a quarter transform gave up waiting for its " \
                      "tensor-core products");                                                   \
  } while (0)

// exact permutational symmetry of the rotated integrals (see k_sym8)
void symmetrize(cudaStream_t st, int n, double* h, double* eri) {
  const int64_t n4 = (int64_t)n * n * n * n;
  HCI_LAUNCH(k_symh, blocks((int64_t)n * n), 256, 0, st)(n, h);
  HCI_LAUNCH(k_sym8, (unsigned)std::min<int64_t>(blocks(n4), 4096), 256, 0, st)(n, eri);
}

}  // namespace

extern "C" hci_status hci_rotate(int norb, const double* kappa, const double* h, const double* eri, double* U,
                                 double* h_out, double* eri_out, void* stream) {
  const int n = norb;
  if (n < 1 || n > HCI_MAXORB) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_rotate: norb=%d outside [1,64]", n);
  if (!kappa || !h || !eri || !U || !h_out || !eri_out)
    return hci_fail(nullptr, HCI_ERR_INVALID, "hci_rotate: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  Scratch S{st};
  const size_t n2 = (size_t)n * n, n4 = n2 * n2;
  double *w1 = S.get(n2), *w2 = S.get(n2), *w3 = S.get(n2), *ds = S.get(8), *t4 = S.get(n4);
  if (!w1 || !w2 || !w3 || !ds || !t4)
    return hci_fail(nullptr, HCI_ERR_NOMEM, "hci_rotate: allocation failed%s",
                    S.left == 0 ? " (injected by HCI_FAIL_ALLOC_AFTER)" : "");
  hci_status s = expm_dev(st, n, kappa, U, w1, w2, w3, ds);
  if (s != HCI_OK) return hci_fail(nullptr, s, "hci_rotate: matrix exponential failed");
  mm(st, n, h, 0, U, 0, w1, 1.0, 0.0);          // h U
  mm(st, n, U, 1, w1, 0, h_out, 1.0, 0.0);      // U^T h U
  QTRANS("hci_rotate", eri, U, t4);
  QTRANS("hci_rotate", t4, U, eri_out);
  QTRANS("hci_rotate", eri_out, U, t4);
  QTRANS("hci_rotate", t4, U, eri_out);
  symmetrize(st, n, h_out, eri_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hci_fail(nullptr, HCI_ERR_CUDA, "hci_rotate: %s", cudaGetErrorString(e));
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hci_fail(nullptr, HCI_ERR_CUDA, "hci_rotate: %s", cudaGetErrorString(e));
  QTRANS_CHECK("hci_rotate");
  return HCI_OK;
}

extern "C" hci_status hci_rotate_backward(int norb, const double* kappa, const double* h, const double* eri,
                                          const double* rdm1, const double* rdm2, double* dh, double* deri,
                                          double* dkappa, void* stream) {
  const int n = norb;
  if (n < 1 || n > HCI_MAXORB)
    return hci_fail(nullptr, HCI_ERR_INVALID, "hci_rotate_backward: norb=%d outside [1,64]", n);
  if (!kappa || !h || !eri || !rdm1 || !rdm2)
    return hci_fail(nullptr, HCI_ERR_INVALID, "hci_rotate_backward: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  Scratch S{st};
  const size_t n2 = (size_t)n * n, n4 = n2 * n2;
  const int m2 = 2 * n;
  double *U = S.get(n2), *Ut = S.get(n2), *I = S.get(n2), *w1 = S.get(n2), *gU = S.get(n2);
  double *b1 = S.get((size_t)m2 * m2), *b2 = S.get((size_t)m2 * m2), *b3 = S.get((size_t)m2 * m2),
         *b4 = S.get((size_t)m2 * m2), *b5 = S.get((size_t)m2 * m2), *ds = S.get(8);
  double *D = S.get(n4), *t4 = S.get(n4);
  if (!U || !Ut || !I || !w1 || !gU || !b1 || !b2 || !b3 || !b4 || !b5 || !ds || !D || !t4)
    return hci_fail(nullptr, HCI_ERR_NOMEM, "hci_rotate_backward: allocation failed%s",
                    S.left == 0 ? " (injected by HCI_FAIL_ALLOC_AFTER)" : "");
  cudaFuncSetAttribute(k_gemm_nt_part, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * NT_CH * 8);
  hci_status s = expm_dev(st, n, kappa, U, w1, b1, b2, ds);
  if (s != HCI_OK) return hci_fail(nullptr, s, "hci_rotate_backward: matrix exponential failed");
  HCI_LAUNCH(k_eye, blocks((int64_t)n2), 256, 0, st)(n, I);
  // U^T as a matrix for the back-transforms: M[a][p] = U[p][a]
  mm(st, n, U, 1, I, 0, Ut, 1.0, 0.0);
  if (dh) {
    mm(st, n, rdm1, 0, U, 1, w1, 1.0, 0.0);     // g1 U^T
    mm(st, n, U, 0, w1, 0, dh, 1.0, 0.0);       // U g1 U^T
  }
  HCI_LAUNCH(k_scale_copy, blocks((int64_t)n4), 256, 0, st)((int64_t)n4, rdm2, 0.5, D);
  if (deri) {
    QTRANS("hci_rotate_backward", D, Ut, t4);
    QTRANS("hci_rotate_backward", t4, Ut, deri);
    QTRANS("hci_rotate_backward", deri, Ut, t4);
    QTRANS("hci_rotate_backward", t4, Ut, deri);
  }
  if (dkappa) {
    // h-part: h U g1^T + h^T U g1
    mm(st, n, h, 0, U, 0, w1, 1.0, 0.0);
    mm(st, n, w1, 0, rdm1, 1, gU, 1.0, 0.0);
    mm(st, n, h, 1, U, 0, w1, 1.0, 0.0);
    mm(st, n, w1, 0, rdm1, 0, gU, 1.0, 1.0);
    // T[y][b][c][d] = sum_qrs U_bq U_cr U_ds D[y][q][r][s]
    double* T = t4;
    QTRANS("hci_rotate_backward", D, I, T);          // (q r s y)
    QTRANS("hci_rotate_backward", T, Ut, D);         // (r s y b)
    QTRANS("hci_rotate_backward", D, Ut, T);         // (s y b c)
    QTRANS("hci_rotate_backward", T, Ut, D);         // (y b c d)
    const int64_t K = (int64_t)n * n * n;
    const int nparts = (int)((K + NT_CH - 1) / NT_CH);
    double* part = S.get((size_t)nparts * n2);
    if (!part)
      return hci_fail(nullptr, HCI_ERR_NOMEM, "hci_rotate_backward: allocation failed%s",
                      S.left == 0 ? " (injected by HCI_FAIL_ALLOC_AFTER)" : "");
    HCI_LAUNCH(k_gemm_nt_part, nparts, 256, (size_t)2 * n * NT_CH * 8, st)(n, K, eri, D, part);
    HCI_LAUNCH(k_sum_parts, blocks((int64_t)n2), 256, 0, st)((int)n2, nparts, part, 4.0, gU);
    // dkappa = L_exp(kappa^T, gU)
    HCI_LAUNCH(k_frechet_block, blocks((int64_t)m2 * m2), 256, 0, st)(n, kappa, gU, b1);
    s = expm_dev(st, m2, b1, b2, b3, b4, b5, ds);
    if (s != HCI_OK) return hci_fail(nullptr, s, "hci_rotate_backward: Frechet exponential failed");
    HCI_LAUNCH(k_upper_right, blocks((int64_t)n2), 256, 0, st)(n, b2, dkappa);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hci_fail(nullptr, HCI_ERR_CUDA, "hci_rotate_backward: %s", cudaGetErrorString(e));
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hci_fail(nullptr, HCI_ERR_CUDA, "hci_rotate_backward: %s", cudaGetErrorString(e));
  QTRANS_CHECK("hci_rotate_backward");
  return HCI_OK;
}

extern "C" hci_status hci_qtrans(int norb, const double* in, const double* M, double* out, int check,
                                 void* stream) {
  const int n = norb;
  if (n < 1 || n > HCI_MAXORB) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_qtrans: norb=%d outside [1,64]", n);
  if (!in || !M || !out) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_qtrans: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  QTRANS("hci_qtrans", in, M, out);
  if (check) QTRANS_CHECK("hci_qtrans");
  return HCI_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free rotation.
//
// Some callers cannot allocate device memory at the time they need the
// rotation: code running inside another framework's memory pool that forbids
// foreign allocations, or a host thread that must not perform a
// cudaMalloc/cudaFree (each may synchronise the device).  For them
// hci_rotate_noalloc computes exactly what hci_rotate computes, with its
// scratch (the n^4 intermediate of the quarter transforms and the work
// matrices of exp(kappa)) in the file-scope device array below instead of
// stream-ordered allocations.  The array is part of this library's module:
// every GPU that loads the library holds it until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int NOALLOC_MAXORB = 32;
constexpr size_t NOALLOC_T4 = (size_t)NOALLOC_MAXORB * NOALLOC_MAXORB * NOALLOC_MAXORB * NOALLOC_MAXORB;
constexpr size_t NOALLOC_M = (size_t)NOALLOC_MAXORB * NOALLOC_MAXORB;
constexpr size_t NOALLOC_DOUBLES = NOALLOC_T4 + 3 * NOALLOC_M + 32;   // 8.02 MiB

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

constexpr int NOALLOC_MAXDEV = 64;
struct NoallocSlot {
  unsigned long long ctx_id = 0;   // context the address was looked up in (0: none)
  double* ptr = nullptr;
};
static NoallocSlot g_noalloc_slot[NOALLOC_MAXDEV];
static std::mutex g_noalloc_mu;

// Identity of the calling thread's current CUDA context (a driver-assigned id
// that is never reused), 0 when it cannot be read.  The driver entry points
// are fetched through the runtime, so the library does not link libcuda.
unsigned long long current_context_id() {
  typedef CUresult (*GetCurrent)(CUcontext*);
  typedef CUresult (*GetId)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
        qa == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(a);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
        qb == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(b);
    cudaGetLastError();
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress (with the device current) once per device and
// context: the cached address is used again only while the same context is
// current, so a device reset or another context gets its own look-up.
hci_status noalloc_scratch(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hci_fail(nullptr, HCI_ERR_CUDA, "hci_rotate_noalloc: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= NOALLOC_MAXDEV)
    return hci_fail(nullptr, HCI_ERR_INVALID, "hci_rotate_noalloc: device %d outside [0,%d)", dev, NOALLOC_MAXDEV);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoallocSlot& slot = g_noalloc_slot[dev];
  unsigned long long id = current_context_id();
  if (!slot.ptr || id == 0 || slot.ctx_id != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return hci_fail(nullptr, HCI_ERR_CUDA, "hci_rotate_noalloc: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
    if (id == 0) id = current_context_id();   // the look-up made the primary context current
    slot.ptr = reinterpret_cast<double*>(p);
    slot.ctx_id = id;
  }
  *out = slot.ptr;
  return HCI_OK;
}

}  // namespace

extern "C" hci_status hci_rotate_noalloc(int norb, const double* kappa, const double* h, const double* eri, double* U,
                                         double* h_out, double* eri_out, void* stream) {
  const int n = norb;
  if (n < 1 || n > NOALLOC_MAXORB)
    return hci_fail(nullptr, HCI_ERR_INVALID,
                    "hci_rotate_noalloc: norb=%d outside [1,%d] (the static scratch holds one %d^4 intermediate)", n,
                    NOALLOC_MAXORB, NOALLOC_MAXORB);
  if (!kappa || !h || !eri || !U || !h_out || !eri_out)
    return hci_fail(nullptr, HCI_ERR_INVALID, "hci_rotate_noalloc: null pointer");
  double* base = nullptr;
  hci_status s = noalloc_scratch(&base);
  if (s != HCI_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // every scratch element read below is written first in the same call, so
  // nothing has to be cleared; calls that overlap on the GPU share the array
  // and race
  double* t4 = base;
  double* w1 = base + NOALLOC_T4;
  double* w2 = w1 + NOALLOC_M;
  double* w3 = w2 + NOALLOC_M;
  double* ds = w3 + NOALLOC_M;
  s = expm_dev(st, n, kappa, U, w1, w2, w3, ds);
  if (s != HCI_OK) return hci_fail(nullptr, s, "hci_rotate_noalloc: matrix exponential failed");
  mm(st, n, h, 0, U, 0, w1, 1.0, 0.0);          // h U
  mm(st, n, U, 1, w1, 0, h_out, 1.0, 0.0);      // U^T h U
  QTRANS("hci_rotate_noalloc", eri, U, t4);
  QTRANS("hci_rotate_noalloc", t4, U, eri_out);
  QTRANS("hci_rotate_noalloc", eri_out, U, t4);
  QTRANS("hci_rotate_noalloc", t4, U, eri_out);
  symmetrize(st, n, h_out, eri_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hci_fail(nullptr, HCI_ERR_CUDA, "hci_rotate_noalloc: %s", cudaGetErrorString(e));
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hci_fail(nullptr, HCI_ERR_CUDA, "hci_rotate_noalloc: %s", cudaGetErrorString(e));
  QTRANS_CHECK("hci_rotate_noalloc");
  return HCI_OK;
}
