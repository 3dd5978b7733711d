// Internal declarations shared by the translation units of libhci.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

#include "../../include/hci.h"

#define HCI_MAXORB 64

// Grow-only device buffer, stream-ordered allocation on the context stream.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Stored connections are kept in segments (one per build or extension of
// the space); a row's first entry is addressed as segment << GRAPH_SEG_SHIFT
// | offset within the segment, and the segment table is handed to kernels by
// value.
constexpr int GRAPH_MAXSEG = 32;
constexpr int GRAPH_SEG_SHIFT = 40;
constexpr int64_t GRAPH_SEG_MASK = ((int64_t)1 << GRAPH_SEG_SHIFT) - 1;
struct SegTab {
  const int32_t* col[GRAPH_MAXSEG];
  const double* val[GRAPH_MAXSEG];
};

// Connection graph of one determinant space (Sec. IV: the Hamiltonian on V
// is evaluated from every single and double excitation linking two
// determinants of V; the same connections feed the RDMs).  Rows and columns
// are internal ids (insertion order).  Both orientations: each row holds all
// of its connections in a pool with per-row slack (segment 0).  One
// orientation: each connected pair is stored once, in the row of the
// determinant with the larger id, one segment per build or extension (a
// grown space only adds rows); H c adds every stored entry to both rows.
struct Graph {
  bool valid = false;
  int64_t nV = 0;
  uint64_t hash = 0;
  int64_t nnz = 0;           // off-diagonal connections, both orientations counted (2 x stored)
  int64_t nstored = 0;       // stored entries, one per connected pair
  int64_t nua = 0, nub = 0;  // distinct alpha / beta strings of the space
  bool half = false;         // one orientation per pair (else both, in a row pool with slack)
  DevBuf rowptr;             // int64 [nV+1] prefix sums of the stored row lengths (internal order)
  DevBuf rowstart;           // int64 [nV] first entry of each row: segment << GRAPH_SEG_SHIFT | offset
  DevBuf rowlen;             // both orientations: int64 [nV] live entries of each row
  DevBuf rowcap;             // both orientations: int64 [nV] slots owned by each row (>= rowlen)
  int64_t pool_used = 0, pool_cap = 0;   // both orientations: slots of the row pool (segment 0)
  DevBuf seg_col[GRAPH_MAXSEG];   // int32 columns (internal ids; one orientation: all below the row's id)
  DevBuf seg_val[GRAPH_MAXSEG];   // double <D_i|H|D_j>
  int nseg = 0;
  DevBuf diag;               // double [nV]
  DevBuf keys;               // copy of the space's keys [nV][2], sorted
  DevBuf keys_int;           // the same keys by internal id (insertion order)
  DevBuf s2i, i2s;           // int32 maps sorted position <-> internal id
  bool direct = false;       // no stored rows: every traversal searches and evaluates the connections again
  int64_t epoch = 0;         // increases with every build or extension
  int64_t parent = -1;       // extension: the epoch it grew from (else -1)
  int64_t nold = 0;          // extension: rows of the space it grew from (ids below nold)
  int64_t tail_entries = 0;  // extension: stored entries in rows nold .. nV-1
  SegTab tab() const {
    SegTab t{};
    for (int k = 0; k < nseg; ++k) {
      t.col[k] = reinterpret_cast<const int32_t*>(seg_col[k].p);
      t.val[k] = reinterpret_cast<const double*>(seg_val[k].p);
    }
    return t;
  }
};

struct Lists {
  bool built = false;
  int n = 0;
  int len_opp = 0, len_same = 0;     // entries per list
  int npair_same = 0;                // n(n-1)/2
  DevBuf opp_mag, opp_tgt;           // [n*n][len_opp] double / uint16 (r | s<<8)
  DevBuf same_mag, same_tgt;         // [npair_same][len_same]
  DevBuf single_bound;               // [n*n] upper bound of |H| for single p->r
  DevBuf list_max;                   // [n*n + npair_same] first (largest) magnitude of each list
  DevBuf f_ref;                      // [2][n][n] single-excitation rows of the aufbau determinant (set at create)
  double max_opp = 0, max_same = 0, max_single = 0;
};

// Scratch of the incremental graph update (V' = V + new determinants).
struct IncScratch {
  DevBuf pos_old, mark, flag, newrows, rpN, cnt, keys_old, s2i_old, grow;
  DevBuf colN, valN, hist, tbase, T, T2, tstart, len, rp_old, col_old, val_old, len_old, cap_old;  // both orientations
  DevBuf scr, stage, roff, ctl, left, samp;   // staged row search
};

// Per-phase CUDA-event timers (enabled by hci_profile).
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t open[HCI_PH_COUNT] = {};
  std::vector<std::array<cudaEvent_t, 2>> pend[HCI_PH_COUNT];
  double ms[HCI_PH_COUNT] = {};
  int64_t count[HCI_PH_COUNT] = {};
};

// Lowest Ritz vectors (and their H products) of the last single-root
// Davidson, in the internal order of the graph epoch they belong to; a
// Davidson on a space grown from that one starts from them.
struct DavKeep {
  bool valid = false;
  int64_t epoch = -1, nV = 0, ld = 0;
  int k = 0;
  DevBuf Q, W;
};

struct hci_ctx {
  int n = 0, na = 0, nb = 0;
  double ecore = 0;
  cudaStream_t st = nullptr;
  DevBuf h, eri;                     // device copies
  DevBuf jk_same, j_opp;             // n^3 tables for single excitations
  Lists lists;
  Graph graph;
  // scratch
  DevBuf s_cand, s_cand2, s_flags, s_scan, s_misc, s_counter, s_hist, s_walkstat, s_items, s_rdmw, s_rdmh;
  DevBuf p2_vals, p2_vals2, p2_ref, p2_src, p2_src2, p2_d, p2_dd;   // perturbative correction
  DevBuf ss_w, ss_draw, ss_draw2, ss_run, ss_src;                 // sampled perturbative correction
  DevBuf g_ua, g_ga, g_ia, g_ub, g_gb, g_ib, g_permb, g_bkeys, g_bkeys2, g_nbr_ptr, g_nbr, g_cnt;
  DevBuf g_bnbr_ptr, g_bnbr, g_costa, g_costb, g_htab, g_hval, g_posb, g_vb, g_ba;
  DevBuf g_nscr;   // padded neighbour lists of the one-pass look-up
  IncScratch inc;
  bool incremental = true;
  int sigma_mode = HCI_SIGMA_AUTO;
  int64_t graph_budget = 0;  // bytes the stored connection pool may take (0: device memory)
  bool direct_fallback = false;
  bool half_fallback = false;
  DevBuf d_vb, d_wb, d_diag, d_small, d_part, d_perm, d_zv, d_rel, d_lock;
  DavKeep dkeep;
  int spin_parity = 0;             // 0, or +1 / -1: states with c(beta,alpha) = p c(alpha,beta) (S_z = 0)
  DevBuf d_partner;                // int32 spin-flip partner of each internal id
  int64_t partner_epoch = -1;      // graph epoch d_partner belongs to
  int nsm = 0;               // streaming multiprocessors of the context's device (grid sizes)
  size_t mem_total = 0;      // device memory of the context's device (bytes)
  size_t l2_bytes = 0;       // L2 cache of the context's device (bytes)
  int half_passes = 0;       // HCI_SIGMA_HALF_PASSES: 1 or 2 forces the one-orientation product's passes (0: by size)
  int64_t fail_alloc_after = -1;  // HCI_FAIL_ALLOC_AFTER: allocations left before one is refused (-1: off)
  int64_t last_candidates = 0;
  int64_t st_counts[HCI_ST_COUNT] = {};
  Prof prof;
  char err[512] = {0};
};

void prof_tic(hci_ctx* ctx, int phase);
void prof_toc(hci_ctx* ctx, int phase);
void prof_release(hci_ctx* ctx);

// Every kernel launch of the library goes through HCI_LAUNCH, which counts it.
extern std::atomic<long long> g_hci_launches;
inline void hci_count_launch() { g_hci_launches.fetch_add(1, std::memory_order_relaxed); }
#define HCI_LAUNCH(k, ...) hci_count_launch(), k<<<__VA_ARGS__>>>

// ----------------------------------------------------------------------------
// error helpers
// ----------------------------------------------------------------------------
hci_status hci_fail(hci_ctx* ctx, hci_status code, const char* fmt, ...);

#define HCI_CUDA(ctx, call)                                                                \
  do {                                                                                     \
    cudaError_t _e = (call);                                                               \
    if (_e != cudaSuccess)                                                                 \
      return hci_fail((ctx), HCI_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,     \
                      cudaGetErrorString(_e));                                             \
  } while (0)

#define HCI_TRY(expr)                 \
  do {                                \
    hci_status _s = (expr);           \
    if (_s != HCI_OK) return _s;      \
  } while (0)

// Ensure buf holds at least `bytes` (contents are NOT preserved on growth).
hci_status ensure_buf(hci_ctx* ctx, DevBuf& b, size_t bytes);
void free_buf(cudaStream_t st, DevBuf& b);

template <class T>
inline T* bp(DevBuf& b) { return reinterpret_cast<T*>(b.p); }

// SM count of the device the last context was created on (152 on GB300);
// grid-stride launches without a context size their grids from it.
extern int g_hci_nsm;
inline int hci_nsm() { return g_hci_nsm > 0 ? g_hci_nsm : 152; }

// Host-side fault injection for tests: the value of the environment variable
// HCI_FAIL_ALLOC_AFTER (k >= 0: the first k allocations succeed, every later
// one is refused as if the device were out of memory), or -1 when unset.
int64_t hci_fail_alloc_env();

// Quarter transform of the integral rotation, out[J][p] = sum_a in[a][J]
// M[a][p] for J < n^3 (qtrans_tc.cu): exact digit products on the bf16
// tensor cores, rounded once to FP64.  qtrans_tc_check() reports (and
// clears) a launch on stream st that gave up waiting for its products (it
// reads a device flag on st and synchronises st).
hci_status qtrans_tc(cudaStream_t st, int n, const double* in, const double* M, double* out);
hci_status qtrans_tc_check(cudaStream_t st);

inline int grid_for(int64_t work, int block, int max_blocks = -1) {
  if (max_blocks < 0) max_blocks = hci_nsm() * 16;
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

// ----------------------------------------------------------------------------
// primitives (prims.cu)
// ----------------------------------------------------------------------------
// Exclusive scan of int64 values in place-free form: out[i] = sum_{j<i} in[j];
// returns the total through *total_dev (device pointer, may be NULL).
hci_status scan_i64(hci_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev);
// Stable LSD radix sort of 128-bit keys (a = high word, b = low word) on
// the low `bits_a` / `bits_b` bits.  Result in keys (tmp is scratch of same size).
hci_status sort_keys(hci_ctx* ctx, uint64_t* keys, uint64_t* tmp, int64_t n, int bits_a, int bits_b);
// the same, carrying one double (vals, with vtmp as scratch) and one int32
// (idx, with itmp as scratch) per key; either may be NULL
hci_status sort_pairs(hci_ctx* ctx, uint64_t* keys, uint64_t* tmp, double* vals, double* vtmp, int32_t* idx,
                      int32_t* itmp, int64_t n, int bits_a, int bits_b);
// 64-bit content hash of a key array (device result).
hci_status hash_keys(hci_ctx* ctx, const uint64_t* keys, int64_t n, uint64_t* hash_host);
// Checks that keys are strictly ascending (device reduction); *ok_host = 1 if sorted.
hci_status check_sorted(hci_ctx* ctx, const uint64_t* keys, int64_t n, int* ok_host);

// graph.cu
hci_status graph_ensure(hci_ctx* ctx, const uint64_t* keys, int64_t nV);
// sigma on vectors in internal order (rows/columns of the cached graph)
hci_status sigma_apply(hci_ctx* ctx, const double* c, double* sigma, int nvec);
// out[i] = sum_j H_ij c_j for the rows i in [r0, nV) of the cached stored
// graph, off-diagonal entries only, for a c that vanishes on those rows
hci_status sigma_tail(hci_ctx* ctx, int64_t r0, const double* c, double* out);
struct RdmAcc;
// off-diagonal RDM contributions of a direct graph (one orientation per pair)
hci_status direct_rdm(hci_ctx* ctx, const double* c, const RdmAcc& R);
// density matrices of the perturbative correction (rdm.cu)
hci_status pt2_rdm_begin(hci_ctx* ctx);
hci_status pt2_rdm_pairs(hci_ctx* ctx, const ulonglong2* V, const double* c, const ulonglong2* tgt, const int32_t* src,
                         const double* d, int64_t m);
hci_status pt2_rdm_finish(hci_ctx* ctx, double* r1dd, double* r2dd, double* r1dc, double* r2dc);
// vectors between the caller's (sorted) order and the graph's internal order
hci_status to_internal(hci_ctx* ctx, const double* sorted, double* internal, int nvec);
hci_status to_sorted(hci_ctx* ctx, const double* internal, double* sorted, int nvec);

// device helpers -------------------------------------------------------------
__device__ __forceinline__ int popc64(uint64_t x) { return __popcll(x); }

// (-1)^(number of set bits of s strictly between orbitals p and r)
__device__ __forceinline__ double exc_phase(uint64_t s, int p, int r) {
  int lo = p < r ? p : r, hi = p < r ? r : p;
  uint64_t mask = ((hi >= 64) ? ~0ull : ((1ull << hi) - 1ull)) & ~((2ull << lo) - 1ull);
  return (__popcll(s & mask) & 1) ? -1.0 : 1.0;
}
