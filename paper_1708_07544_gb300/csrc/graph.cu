// Connection graph of a determinant space and the FP64 sigma H c.
//
// Sec. IV: the Hamiltonian on V is built from all pairs of determinants of V
// that differ by a single or double excitation.  Instead of generating the
// ~N^2 n^2 excitations of each row and looking them up, the determinants are
// grouped by alpha string (V is sorted by (alpha, beta)) and by beta string
// (a second, beta-major order), and connections are found by XOR/popcount
// scans:
//   (A) same alpha string, beta differs by 1 or 2 electrons;
//   (B) same beta string, alpha differs by 1 or 2 electrons;
//   (C) alpha differs by a single (via the single-excitation neighbours of
//       each distinct alpha string) and beta differs by a single.
// The three sets are disjoint.  Two stored forms (hci_set_sigma_mode):
//   both orientations: every row holds all of its connections in a row pool
//     with slack (12 B per ordered pair); H c is a pure gather over the
//     rows, and growing the space appends the new rows' transposes to the
//     old rows in place;
//   one orientation: each connected pair is stored once, in the row of the
//     determinant with the larger internal id (ids are insertion order), in
//     one segment per build or extension (half the memory; growing the
//     space only appends rows), and H c adds each entry to both of its rows
//     (a row sum plus an FP64 atomic scatter into the other row).
#include <algorithm>
#include <vector>

#include "hci_internal.cuh"
#include "rdm_acc.cuh"

namespace {

constexpr int G_WARPS = 8;
// blocks of the row search: six per SM, all resident at 40 registers
inline int rows_grid(const hci_ctx* ctx) { return ctx->nsm * 6; }
constexpr int64_t ROW_SCR = 32768;   // scratch entries per warp of the staged row search
constexpr int64_t ROW_SAMPLE = 2048; // rows counted to size the staging buffer

__device__ __forceinline__ bool key_less(ulonglong2 a, ulonglong2 b) {
  return a.x < b.x || (a.x == b.x && a.y < b.y);
}
__device__ __forceinline__ int64_t lower_bound_k(const ulonglong2* __restrict__ arr, int64_t n, ulonglong2 key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (key_less(arr[mid], key)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int64_t lower_bound_u(const uint64_t* __restrict__ arr, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (arr[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// grouping
// ---------------------------------------------------------------------------
// word = 0: group by .x (alpha) of keys; word = 1: by .x of swapped keys
__global__ void k_run_flags(const ulonglong2* __restrict__ keys, int64_t n, int64_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || keys[i].x != keys[i - 1].x) ? 1 : 0;
}

// group index per element, unique strings and group starts
__global__ void k_groups(const ulonglong2* __restrict__ keys, int64_t n, const int64_t* __restrict__ flag,
                         const int64_t* __restrict__ excl, int32_t* __restrict__ gidx, uint64_t* __restrict__ uniq,
                         int64_t* __restrict__ start) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t g = excl[i] + flag[i] - 1;
    gidx[i] = (int32_t)g;
    if (flag[i]) {
      uniq[g] = keys[i].x;
      start[g] = i;
    }
  }
}

__global__ void k_set_last(int64_t* start, const int64_t* ngroups_dev, int64_t n) {
  start[*ngroups_dev] = n;
}

__global__ void k_store_at(int64_t* arr, int64_t idx, const int64_t* val) { arr[idx] = *val; }

__global__ void k_swap_keys(const ulonglong2* __restrict__ in, int64_t n, ulonglong2* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 k = in[i];
    out[i] = make_ulonglong2(k.y, k.x);
  }
}

// permb[k] = index in V of the k-th determinant in beta-major order;
// ib[permb[k]] = beta group of position k
__global__ void k_perm_b(const ulonglong2* __restrict__ bkeys, int64_t n, const ulonglong2* __restrict__ V,
                         const int32_t* __restrict__ bgroup_of_pos, int32_t* __restrict__ permb,
                         int32_t* __restrict__ ib, int32_t* __restrict__ posb, uint64_t* __restrict__ ba) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 s = bkeys[k];
    int64_t j = lower_bound_k(V, n, make_ulonglong2(s.y, s.x));
    permb[k] = (int32_t)j;
    ib[j] = bgroup_of_pos[k];
    posb[j] = (int32_t)k;
    ba[k] = s.y;
  }
}

__global__ void k_pack_beta(const ulonglong2* __restrict__ V, int64_t n, uint64_t* __restrict__ vb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    vb[i] = V[i].y;
}

// Open-addressing hash set of the distinct strings (value = group index),
// linear probing; table size is a power of two >= 2 x entries, so probing
// always ends at an empty slot.
constexpr uint64_t HASH_EMPTY = ~0ull;

__device__ __forceinline__ uint64_t hash_str(uint64_t x) {
  x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33;
  return x;
}

__global__ void k_hash_insert(const uint64_t* __restrict__ u, int64_t nu, unsigned long long* __restrict__ tab,
                              int32_t* __restrict__ val, uint64_t mask) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nu; g += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = u[g];
    uint64_t h = hash_str(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      const unsigned long long prev = atomicCAS(&tab[h], (unsigned long long)HASH_EMPTY, (unsigned long long)key);
      if (prev == HASH_EMPTY || prev == key) {
        val[h] = (int32_t)g;
        break;
      }
      h = (h + 1) & mask;
    }
  }
}

__device__ __forceinline__ int32_t hash_find(const unsigned long long* __restrict__ tab, const int32_t* __restrict__ val,
                                             uint64_t mask, uint64_t key) {
  uint64_t h = hash_str(key) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const unsigned long long t = tab[h];
    if (t == key) return val[h];
    if (t == HASH_EMPTY) return -1;
    h = (h + 1) & mask;
  }
  return -1;
}

// ---------------------------------------------------------------------------
// Slater-Condon element <D_i|H|D_j> for a known connection
// ---------------------------------------------------------------------------
struct HamView {
  int n;
  const double* h;
  const double* eri;
  const double* jk_same;   // [p][r][k] (pr|kk) - (pk|kr)
  const double* j_opp;     // [p][r][k] (pr|kk)
  const double* f_ref;     // [spin][p][r] single p->r of the aufbau determinant
  uint64_t ref_a, ref_b;   // aufbau alpha / beta strings
};

__device__ __forceinline__ double eri4(const HamView& H, int p, int r, int q, int s) {
  return H.eri[(((int64_t)p * H.n + r) * H.n + q) * H.n + s];
}

// single p->r in spin string sj (other spin string oj), both of D_j; spin 0
// = alpha.  h_pr + sum_{k in sj} [(pr|kk) - (pk|kr)] + sum_{k in oj} (pr|kk)
// is taken as the aufbau determinant's value plus the terms of the orbitals
// where sj and oj differ from the aufbau strings (a few for a selected
// determinant, instead of a pass over all n orbitals).
__device__ __forceinline__ double single_el(const HamView& H, uint64_t sj, uint64_t oj, int p, int r, int spin) {
  const uint64_t rs = spin ? H.ref_b : H.ref_a, ro = spin ? H.ref_a : H.ref_b;
  double v = H.f_ref[((int64_t)spin * H.n + p) * H.n + r];
  const double* js = H.jk_same + ((int64_t)p * H.n + r) * H.n;
  const double* jo = H.j_opp + ((int64_t)p * H.n + r) * H.n;
  for (uint64_t m = sj & ~rs; m; m &= m - 1) v += js[__ffsll((long long)m) - 1];
  for (uint64_t m = rs & ~sj; m; m &= m - 1) v -= js[__ffsll((long long)m) - 1];
  for (uint64_t m = oj & ~ro; m; m &= m - 1) v += jo[__ffsll((long long)m) - 1];
  for (uint64_t m = ro & ~oj; m; m &= m - 1) v -= jo[__ffsll((long long)m) - 1];
  return exc_phase(sj, p, r) * v;
}

__device__ __forceinline__ double same_double_el(const HamView& H, uint64_t sj, uint64_t x) {
  uint64_t holes = sj & x, parts = x & ~sj;
  int p = __ffsll((long long)holes) - 1; holes &= holes - 1;
  int q = __ffsll((long long)holes) - 1;
  int r = __ffsll((long long)parts) - 1; parts &= parts - 1;
  int s = __ffsll((long long)parts) - 1;
  double s1 = exc_phase(sj, p, r);
  uint64_t t = sj ^ (1ull << p) ^ (1ull << r);
  double s2 = exc_phase(t, q, s);
  return s1 * s2 * (eri4(H, p, r, q, s) - eri4(H, p, s, q, r));
}

__device__ double connection_el(const HamView& H, ulonglong2 ki, ulonglong2 kj) {
  uint64_t xa = ki.x ^ kj.x, xb = ki.y ^ kj.y;
  int da = __popcll(xa), db = __popcll(xb);
  if (da == 0) {
    if (db == 2) {
      int p = __ffsll((long long)(kj.y & xb)) - 1, r = __ffsll((long long)(ki.y & xb)) - 1;
      return single_el(H, kj.y, kj.x, p, r, 1);
    }
    return same_double_el(H, kj.y, xb);
  }
  if (db == 0) {
    if (da == 2) {
      int p = __ffsll((long long)(kj.x & xa)) - 1, r = __ffsll((long long)(ki.x & xa)) - 1;
      return single_el(H, kj.x, kj.y, p, r, 0);
    }
    return same_double_el(H, kj.x, xa);
  }
  int p = __ffsll((long long)(kj.x & xa)) - 1, r = __ffsll((long long)(ki.x & xa)) - 1;
  int q = __ffsll((long long)(kj.y & xb)) - 1, s = __ffsll((long long)(ki.y & xb)) - 1;
  return exc_phase(kj.x, p, r) * exc_phase(kj.y, q, s) * eri4(H, p, r, q, s);
}

// ---------------------------------------------------------------------------
// row traversal: (A) alpha group, (B) beta group, (C) alpha-single x beta-single
// ---------------------------------------------------------------------------
struct GraphArgs {
  const ulonglong2* V;     // alpha-major keys
  const ulonglong2* bk;    // beta-major swapped keys (beta, alpha)
  int64_t nV;
  int n, na, nb;
  const int32_t* ia;       // alpha group of each det
  const int64_t* ga;       // alpha group starts [nua+1]
  const int32_t* ib;       // beta group of each det
  const int64_t* gb;       // beta group starts (beta-major positions) [nub+1]
  const int32_t* permb;    // beta-major position -> det
  const uint64_t* vb;      // beta string of each det, alpha-major order (packed)
  const uint64_t* ba;      // alpha string of each det, beta-major order (packed)
  const int32_t* posb;     // det -> its beta-major position
  const int64_t* anbr_ptr; // single-excitation neighbours of each distinct alpha string
  const int32_t* anbr;
  const int64_t* bnbr_ptr; // ... of each distinct beta string
  const int32_t* bnbr;
  const int64_t* costa;    // cost of the alpha-side (C) search per distinct alpha string
  const int64_t* costb;
  const int32_t* rowlist;  // rows to process (nullptr: all rows, in order)
  int64_t nrows;
  const int64_t* rowptr;   // fill pass: output offset per processed row
  int32_t* col;
  double* val;
  int64_t* rowcnt;         // count / staged pass: entries per processed row
  int32_t* scr;            // staged pass: scr_cap entries of scratch per warp of the grid
  int64_t scr_cap;
  int32_t* stage;          // staged pass: rows, each contiguous, at rowoff[q]
  int64_t stage_cap;
  int64_t* rowoff;
  unsigned long long* stage_ctl;  // [0] next free staging entry, [1] rows left to the fill pass
  const int32_t* s2i;      // sorted position -> internal id (columns are stored as internal ids)
  int lower;               // one-orientation form: a row keeps the connections with a smaller id
  unsigned long long* queue;
  HamView H;
  // direct traversals (no stored rows), vectors by sorted position
  const double* dc;             // input vector
  double* dsig;                 // sigma: output
  const double* ddiag;          // sigma: diagonal elements
  unsigned long long* dnnz;     // sigma: connections visited (may be null)
  RdmAcc R;                     // RDMs: accumulators
};

// A group of size m is scanned when that is cheaper than L binary searches.
__device__ __forceinline__ bool use_lookup(int64_t m, int L) {
  int lg = 64 - __clzll((long long)(m + 1));
  return m > (int64_t)L * lg;
}

// Row search modes: count only, fill at a known offset, or staged fill
// (into the warp's scratch, capped at scr_cap entries, still counting past it).
// With A.lower these three keep only the connections j whose internal id is
// below the row's (the one-orientation form).  Direct traversals evaluate
// every connection as it is found: ROWS_SIGMA adds H_ij c_j into the row's
// sum, ROWS_RDM accumulates <D_i| op |D_j> c_i c_j for j > i (the other
// orientation is added as the transpose).
constexpr int ROWS_COUNT = 0, ROWS_FILL = 1, ROWS_STAGED = 2, ROWS_SIGMA = 3, ROWS_RDM = 4;

// per-row state: row (sorted position), its internal id, c_i, partial sum
struct RowAcc {
  int64_t i;
  int32_t id;
  double ci;
  double acc;
};

template <int MODE>
__device__ __forceinline__ void visit(const GraphArgs& A, ulonglong2 ki, int64_t j, bool ok, int64_t& w,
                                      int32_t* out, RowAcc& ra) {
  const int lane = threadIdx.x & 31;
  int32_t id = 0;
  if (MODE == ROWS_COUNT || MODE == ROWS_FILL || MODE == ROWS_STAGED) {
    if (ok && (A.lower || MODE != ROWS_COUNT)) {
      id = A.s2i[j];
      if (A.lower) ok = id < ra.id;
    }
  }
  unsigned m = __ballot_sync(0xffffffffu, ok);
  if ((MODE == ROWS_FILL || MODE == ROWS_STAGED) && ok) {
    int64_t pos = w + __popc(m & ((1u << lane) - 1u));
    if (MODE == ROWS_FILL || pos < A.scr_cap) out[pos] = id;
  }
  if (MODE == ROWS_SIGMA && ok) ra.acc = fma(connection_el(A.H, ki, A.V[j]), A.dc[j], ra.acc);
  if (MODE == ROWS_RDM && ok && j > ra.i) {
    const double cc = ra.ci * A.dc[j];
    if (cc != 0.0) rdm_accumulate(A.R, A.n, ki, A.V[j], cc);
  }
  w += __popc(m);
}

// (C) from one side.  BETA == false: neighbours are alpha strings, groups are
// alpha groups (members j = position, other-spin value V[j].y); BETA == true:
// neighbours are beta strings, groups live in beta-major order (members
// j = permb[pos], other-spin value bk[pos].y).  Small groups are scanned
// (flattened, 32 groups at a time); large groups are probed with binary
// searches for the L single excitations of the other-spin string.
template <int MODE, bool BETA>
__device__ __forceinline__ void mixed_side(const GraphArgs& A, ulonglong2 ki, int g, int64_t& w, int32_t* out,
                                           int64_t* s_start, int64_t* s_pref, int64_t* s_size, const int* occ_o,
                                           const int* vir_o, int nocc_o, int nvir_o, RowAcc& ra) {
  const int lane = threadIdx.x & 31;
  const int64_t* ptr = BETA ? A.bnbr_ptr : A.anbr_ptr;
  const int32_t* nbr = BETA ? A.bnbr : A.anbr;
  const int64_t* gs = BETA ? A.gb : A.ga;
  const uint64_t mine = BETA ? ki.x : ki.y;     // other-spin string of row i
  const int L = nocc_o * nvir_o;
  const int64_t nb0 = ptr[g], nb1 = ptr[g + 1];
  for (int64_t c0 = nb0; c0 < nb1; c0 += 32) {
    const int64_t cidx = c0 + lane;
    int64_t st = 0, sz = 0;
    bool look = false;
    if (cidx < nb1) {
      const int gg = nbr[cidx];
      st = gs[gg];
      sz = gs[gg + 1] - st;
      look = use_lookup(sz, L);
    }
    const int64_t ssz = look ? 0 : sz;
    int64_t inc = ssz;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    s_start[lane] = st;
    s_size[lane] = sz;
    s_pref[lane + 1] = inc;
    if (lane == 0) s_pref[0] = 0;
    __syncwarp();
    const int64_t total = s_pref[32];
    for (int64_t v0 = 0; v0 < total; v0 += 32) {
      const int64_t v = v0 + lane;
      bool ok = false;
      int64_t j = -1;
      if (v < total) {
        int lo = 0, hi = 31;
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (s_pref[mid] <= v) lo = mid;
          else hi = mid - 1;
        }
        const int64_t pos = s_start[lo] + (v - s_pref[lo]);
        uint64_t other;
        if (BETA) { j = A.permb[pos]; other = A.ba[pos]; }
        else { j = pos; other = A.vb[pos]; }
        ok = __popcll(mine ^ other) == 2;
      }
      visit<MODE>(A, ki, j, ok, w, out, ra);
    }
    unsigned lk = __ballot_sync(0xffffffffu, look);
    while (lk) {
      const int src = __ffs(lk) - 1;
      lk &= lk - 1;
      const int64_t st2 = s_start[src], sz2 = s_size[src];
      for (int t0 = 0; t0 < L; t0 += 32) {
        const int t = t0 + lane;
        bool ok = false;
        int64_t j = -1;
        if (t < L) {
          const uint64_t want = mine ^ (1ull << occ_o[t / nvir_o]) ^ (1ull << vir_o[t % nvir_o]);
          int64_t lo = 0, hi = sz2;
          while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            const uint64_t x = BETA ? A.ba[st2 + mid] : A.vb[st2 + mid];
            if (x < want) lo = mid + 1;
            else hi = mid;
          }
          if (lo < sz2) {
            const uint64_t x = BETA ? A.ba[st2 + lo] : A.vb[st2 + lo];
            if (x == want) { ok = true; j = BETA ? A.permb[st2 + lo] : st2 + lo; }
          }
        }
        visit<MODE>(A, ki, j, ok, w, out, ra);
      }
    }
    __syncwarp();
  }
}

__device__ __forceinline__ int occ_vir_lists(uint64_t s, int n, int* occ, int* vir) {
  const int lane = threadIdx.x & 31;
  int bo = 0, bv = 0;
  for (int p0 = 0; p0 < n; p0 += 32) {
    const int p = p0 + lane;
    const bool in = p < n;
    const bool o = in && ((s >> p) & 1ull);
    const unsigned mo = __ballot_sync(0xffffffffu, o);
    const unsigned mv = __ballot_sync(0xffffffffu, in && !o);
    const unsigned lt = (1u << lane) - 1u;
    if (o) occ[bo + __popc(mo & lt)] = p;
    if (in && !o) vir[bv + __popc(mv & lt)] = p;
    bo += __popc(mo);
    bv += __popc(mv);
  }
  __syncwarp();
  return bo;
}

// One warp per row taken from a queue.  ROWS_STAGED: the row goes to the
// warp's scratch; at its end one atomic reserves the row's range of the
// staging buffer and the row is copied there (rowoff[q] = its start, or -1
// when the row outgrew the scratch or the staging buffer; rowcnt[q] is
// exact either way).
template <int MODE>
__global__ void __launch_bounds__(G_WARPS * 32) k_rows(GraphArgs A) {
  __shared__ int64_t s_start[G_WARPS][32];
  __shared__ int64_t s_size[G_WARPS][32];
  __shared__ int64_t s_pref[G_WARPS][33];
  __shared__ int s_occ[G_WARPS][HCI_MAXORB];
  __shared__ int s_vir[G_WARPS][HCI_MAXORB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  while (true) {
    unsigned long long qi = 0;
    if (lane == 0) qi = atomicAdd(A.queue, 1ull);
    const int64_t q = (int64_t)__shfl_sync(0xffffffffu, qi, 0);
    if (q >= A.nrows) break;
    const int64_t i = A.rowlist ? (int64_t)A.rowlist[q] : q;
    const ulonglong2 ki = A.V[i];
    int64_t w = MODE == ROWS_FILL ? A.rowptr[q] : 0;
    int32_t* out = MODE == ROWS_FILL ? A.col
                   : MODE == ROWS_STAGED ? A.scr + (int64_t)(blockIdx.x * G_WARPS + wid) * A.scr_cap
                                         : nullptr;
    RowAcc ra{i, A.s2i[i], (MODE == ROWS_SIGMA || MODE == ROWS_RDM) ? A.dc[i] : 0.0, 0.0};
    // (A) same alpha string
    {
      const int g = A.ia[i];
      const int64_t b = A.ga[g], e = A.ga[g + 1];
      for (int64_t j0 = b; j0 < e; j0 += 64) {
        const int64_t j = j0 + lane, j2 = j + 32;
        const uint64_t x1 = j < e ? A.vb[j] : 0ull, x2 = j2 < e ? A.vb[j2] : 0ull;
        bool ok = false, ok2 = false;
        if (j < e && j != i) {
          const int d = __popcll(ki.y ^ x1);
          ok = d == 2 || d == 4;
        }
        if (j2 < e && j2 != i) {
          const int d = __popcll(ki.y ^ x2);
          ok2 = d == 2 || d == 4;
        }
        visit<MODE>(A, ki, j, ok, w, out, ra);
        if (j0 + 32 < e) visit<MODE>(A, ki, j2, ok2, w, out, ra);
      }
    }
    // (B) same beta string
    {
      const int g = A.ib[i];
      const int64_t b = A.gb[g], e = A.gb[g + 1];
      const int64_t mypos = A.posb[i];
      for (int64_t k0 = b; k0 < e; k0 += 64) {
        const int64_t k = k0 + lane, k2 = k + 32;
        const uint64_t x1 = k < e ? A.ba[k] : 0ull, x2 = k2 < e ? A.ba[k2] : 0ull;
        bool ok = false, ok2 = false;
        if (k < e && k != mypos) {
          const int d = __popcll(ki.x ^ x1);
          ok = d == 2 || d == 4;
        }
        if (k2 < e && k2 != mypos) {
          const int d = __popcll(ki.x ^ x2);
          ok2 = d == 2 || d == 4;
        }
        const int64_t j = ok ? (int64_t)A.permb[k] : -1;
        visit<MODE>(A, ki, j, ok, w, out, ra);
        if (k0 + 32 < e) {
          const int64_t j2 = ok2 ? (int64_t)A.permb[k2] : -1;
          visit<MODE>(A, ki, j2, ok2, w, out, ra);
        }
      }
    }
    // (C) single in alpha and single in beta, from the cheaper side
    {
      const int ga_i = A.ia[i], gb_i = A.ib[i];
      if (A.costa[ga_i] <= A.costb[gb_i]) {
        const int no = occ_vir_lists(ki.y, A.n, s_occ[wid], s_vir[wid]);
        mixed_side<MODE, false>(A, ki, ga_i, w, out, s_start[wid], s_pref[wid], s_size[wid], s_occ[wid],
                                s_vir[wid], no, A.n - no, ra);
      } else {
        const int no = occ_vir_lists(ki.x, A.n, s_occ[wid], s_vir[wid]);
        mixed_side<MODE, true>(A, ki, gb_i, w, out, s_start[wid], s_pref[wid], s_size[wid], s_occ[wid],
                               s_vir[wid], no, A.n - no, ra);
      }
    }
    if (MODE == ROWS_COUNT && lane == 0) A.rowcnt[q] = w;
    if (MODE == ROWS_SIGMA) {
      double a = ra.acc;
      for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) {
        A.dsig[i] = fma(A.ddiag[i], ra.ci, a);
        if (A.dnnz) atomicAdd(A.dnnz, (unsigned long long)w);
      }
    }
    if (MODE == ROWS_STAGED) {
      __syncwarp();
      int64_t base = -1;
      if (lane == 0) {
        A.rowcnt[q] = w;
        if (w <= A.scr_cap) {
          const int64_t b = (int64_t)atomicAdd(A.stage_ctl, (unsigned long long)w);
          if (b + w <= A.stage_cap) base = b;
        }
        if (base < 0) atomicAdd(A.stage_ctl + 1, 1ull);
        A.rowoff[q] = base;
      }
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= 0)
        for (int64_t t = lane; t < w; t += 32) A.stage[base + t] = out[t];
      __syncwarp();
    }
  }
}

// rows[t] = list[t * n / ns], an evenly strided sample of ns entries of list
__global__ void k_stride_sample(const int32_t* __restrict__ list, int64_t n, int64_t ns, int32_t* __restrict__ rows) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ns) rows[t] = list[t * n / ns];
}

// Staged rows placed: row q (rowoff[q] >= 0) copied from the staging buffer
// to [rp[q], rp[q] + len) of col, len = lens[q] (or rp[q+1] - rp[q] when
// lens is NULL, a dense CSR), one warp per row.
__global__ void k_copy_staged(const int64_t* __restrict__ rowoff, const int64_t* __restrict__ rp,
                              const int64_t* __restrict__ lens, int64_t nrows, const int32_t* __restrict__ stage,
                              int32_t* __restrict__ col) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp; q < nrows; q += nwarps) {
    const int64_t off = rowoff[q];
    if (off < 0) continue;
    const int64_t b = rp[q], len = lens ? lens[q] : rp[q + 1] - b;
    for (int64_t t = lane; t < len; t += 32) col[b + t] = stage[off + t];
  }
}

// rows the staged pass could not keep: their ids and CSR offsets, for the
// fill pass (any order: each row is written at its own offset)
__global__ void k_collect_left(const int64_t* __restrict__ rowoff, const int64_t* __restrict__ rp,
                               const int32_t* __restrict__ rowlist, int64_t nrows,
                               unsigned long long* __restrict__ counter, int32_t* __restrict__ left_rows,
                               int64_t* __restrict__ left_off) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nrows; q += (int64_t)gridDim.x * blockDim.x)
    if (rowoff[q] < 0) {
      const unsigned long long m = atomicAdd(counter, 1ull);
      left_rows[m] = rowlist[q];
      left_off[m] = rp[q];
    }
}

// Matrix elements of filled rows (the search only records the columns):
// row q holds entries [start[q], start[q] + len) of col/val, with
// len = start[q+1] - start[q] (DENSE) or lens[q]; four entries per lane in
// flight.
template <bool DENSE>
__global__ void __launch_bounds__(256) k_row_values(const int32_t* __restrict__ rowlist, int64_t nrows,
                                                    const int64_t* __restrict__ start,
                                                    const int64_t* __restrict__ lens, const int32_t* __restrict__ col,
                                                    double* __restrict__ val, const ulonglong2* __restrict__ Vrow,
                                                    const ulonglong2* __restrict__ V, HamView H) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp; q < nrows; q += nwarps) {
    const int64_t i = rowlist ? (int64_t)rowlist[q] : q;
    const ulonglong2 ki = Vrow[i];
    const int64_t b = start[q];
    const int64_t len = DENSE ? start[q + 1] - b : lens[q];
    int64_t k = lane;
    for (; k + 96 < len; k += 128) {
      const ulonglong2 k0 = V[col[b + k]], k1 = V[col[b + k + 32]], k2 = V[col[b + k + 64]],
                       k3 = V[col[b + k + 96]];
      val[b + k] = connection_el(H, ki, k0);
      val[b + k + 32] = connection_el(H, ki, k1);
      val[b + k + 64] = connection_el(H, ki, k2);
      val[b + k + 96] = connection_el(H, ki, k3);
    }
    for (; k < len; k += 32) val[b + k] = connection_el(H, ki, V[col[b + k]]);
  }
}

// single-excitation neighbours (within the distinct strings) of each
// distinct string with nocc electrons; count pass (out == nullptr) or fill
// pass.  The nocc * (n - nocc) occupied -> empty pairs are enumerated from
// per-warp occupied / empty lists, p-major, so each list is in (p, r) order.
// With scr, the count pass also writes string g's list at scr + g L (L =
// nocc (n - nocc), its largest possible length), for k_compact_nbrs.
__global__ void __launch_bounds__(256) k_alpha_nbrs(int n, int nocc, const uint64_t* __restrict__ ua, int64_t nua,
                                                    const int64_t* __restrict__ ptr, int64_t* __restrict__ cnt,
                                                    int32_t* __restrict__ out,
                                                    const unsigned long long* __restrict__ tab,
                                                    const int32_t* __restrict__ tval, uint64_t mask,
                                                    int32_t* __restrict__ scr) {
  __shared__ int s_occ[8][HCI_MAXORB];
  __shared__ int s_vir[8][HCI_MAXORB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nvir = n - nocc, L = nocc * nvir;
  for (int64_t g = warp; g < nua; g += nwarps) {
    const uint64_t s = ua[g];
    occ_vir_lists(s, n, s_occ[wid], s_vir[wid]);
    int64_t w = out ? ptr[g] : 0;
    int64_t c = 0;
    for (int t0 = 0; t0 < L; t0 += 32) {
      const int t = t0 + lane;
      int32_t idx = -1;
      if (t < L) idx = hash_find(tab, tval, mask, s ^ (1ull << s_occ[wid][t / nvir]) ^ (1ull << s_vir[wid][t % nvir]));
      const bool hit = idx >= 0;
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (out && hit) out[w + c + __popc(m & ((1u << lane) - 1u))] = idx;
      if (scr && hit) scr[g * L + c + __popc(m & ((1u << lane) - 1u))] = idx;
      c += __popc(m);
    }
    if (!out && lane == 0) cnt[g] = c;
    __syncwarp();
  }
}

// list of string g from its padded slot scr + g L to out + ptr[g]
__global__ void __launch_bounds__(256) k_compact_nbrs(const int32_t* __restrict__ scr, int L,
                                                      const int64_t* __restrict__ ptr, int64_t nua,
                                                      int32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = warp; g < nua; g += nwarps) {
    const int64_t b = ptr[g], len = ptr[g + 1] - b;
    for (int64_t k = lane; k < len; k += 32) out[b + k] = scr[g * L + k];
  }
}

// cost[u] = sum over the neighbours v of string u of min(scan, lookup) cost
__global__ void k_nbr_cost(const int64_t* __restrict__ ptr, const int32_t* __restrict__ nbr,
                           const int64_t* __restrict__ gs, int64_t nu, int L, int64_t* __restrict__ cost) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < nu; u += nwarps) {
    int64_t c = 0;
    for (int64_t k = ptr[u] + lane; k < ptr[u + 1]; k += 32) {
      const int g = nbr[k];
      const int64_t m = gs[g + 1] - gs[g];
      const int lg = 64 - __clzll((long long)(m + 1));
      c += use_lookup(m, L) ? (int64_t)L * lg : m;
    }
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cost[u] = c;
  }
}

// ---------------------------------------------------------------------------
// incremental update: V' = V + N (V's keys all present in V')
// ---------------------------------------------------------------------------
__global__ void k_find_old(const ulonglong2* __restrict__ oldk, int64_t nold, const ulonglong2* __restrict__ V,
                           int64_t nV, int64_t* __restrict__ pos_old, int64_t* __restrict__ mark,
                           unsigned long long* __restrict__ missing) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nold; i += (int64_t)gridDim.x * blockDim.x) {
    const ulonglong2 k = oldk[i];
    const int64_t p = lower_bound_k(V, nV, k);
    if (p < nV && V[p].x == k.x && V[p].y == k.y) {
      pos_old[i] = p;
      mark[p] = 1;
    } else {
      pos_old[i] = -1;
      atomicAdd(missing, 1ull);
    }
  }
}

__global__ void k_not(const int64_t* __restrict__ mark, int64_t n, int64_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = 1 - mark[i];
}

__global__ void k_compact_idx(const int64_t* __restrict__ flag, const int64_t* __restrict__ pos, int64_t n,
                              int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) out[pos[i]] = (int32_t)i;
}

// rows of V' appended after the nold rows already stored: row nold + q has
// rp[q+1] - rp[q] entries starting at offset rp[q] of segment seg, and the
// prefix continues from base (rp[nrows] = the segment's size); with
// nold = 0, base = 0 and rp = rowptr this writes the table of a fresh graph
__global__ void k_append_rows(int64_t nold, int64_t nrows, const int64_t* rp, int64_t base, int seg,
                              int64_t* rowptr, int64_t* __restrict__ rowstart) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q <= nrows; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = rp[q];
    rowptr[nold + q] = base + o;
    if (q < nrows) rowstart[nold + q] = ((int64_t)seg << GRAPH_SEG_SHIFT) | o;
  }
}

// per new row: number of entries whose column is an old determinant; also
// the histogram of those columns (entries to append to old rows)
__global__ void k_count_old_cols(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t nrows,
                                 int64_t nold, int64_t* __restrict__ cnt, int64_t* __restrict__ hist) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp; q < nrows; q += nwarps) {
    int64_t c = 0;
    for (int64_t k = rp[q] + lane; k < rp[q + 1]; k += 32) {
      const int32_t j = col[k];
      if (j < nold) {
        ++c;
        atomicAdd((unsigned long long*)&hist[j], 1ull);
      }
    }
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[q] = c;
  }
}

// T records {x = old column (row to append to) | emitting new row q << 32,
// y = entry index in the new rows' CSR}, written in CSR order
// (deterministic); the sort keys on the low 32 bits of x only
__global__ void k_emit_T(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t nrows,
                         int64_t nold, const int64_t* __restrict__ base, ulonglong2* __restrict__ T) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp; q < nrows; q += nwarps) {
    int64_t w = base[q];
    for (int64_t k0 = rp[q]; k0 < rp[q + 1]; k0 += 32) {
      const int64_t k = k0 + lane;
      bool ok = false;
      int32_t j = 0;
      if (k < rp[q + 1]) {
        j = col[k];
        ok = j < nold;
      }
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (ok)
        T[w + __popc(m & ((1u << lane) - 1u))] = make_ulonglong2((uint64_t)j | ((uint64_t)q << 32), (uint64_t)k);
      w += __popc(m);
    }
  }
}

// ---------------------------------------------------------------------------
// row pool: each row owns [rowstart, rowstart + rowcap) of the col/val
// pools; rowlen <= rowcap entries are live.  Slack lets later updates append
// in place; rows that outgrow it move to the end of the pool.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t slack_cap(int64_t len) { return len + len / 4 + 8; }

__global__ void k_caps(const int64_t* __restrict__ len, int64_t n, int64_t* __restrict__ cap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    cap[i] = slack_cap(len[i]);
}

// Plan of V' = V + N: new length of every row, its capacity, whether it stays
// (start2 = old start) or needs a new range of `need` entries (start2 = -1).
__global__ void k_plan_rows(const int64_t* __restrict__ start_old, const int64_t* __restrict__ len_old,
                            const int64_t* __restrict__ cap_old, int64_t nold, const int64_t* __restrict__ rpN,
                            int64_t nnew, const int64_t* __restrict__ hist, int repack, int64_t* __restrict__ start2,
                            int64_t* __restrict__ len2, int64_t* __restrict__ cap2, int64_t* __restrict__ need) {
  const int64_t tot = nold + nnew;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < nold) {
      const int64_t L = len_old[t] + hist[t];
      len2[t] = L;
      if (!repack && L <= cap_old[t]) {
        start2[t] = start_old[t];
        cap2[t] = cap_old[t];
        need[t] = 0;
      } else {
        start2[t] = -1;
        cap2[t] = slack_cap(L);
        need[t] = cap2[t];
      }
    } else {
      const int64_t q = t - nold;
      const int64_t L = rpN[q + 1] - rpN[q];
      len2[t] = L;
      start2[t] = -1;
      cap2[t] = slack_cap(L);
      need[t] = cap2[t];
    }
  }
}

__global__ void k_assign_starts(int64_t* __restrict__ start2, const int64_t* __restrict__ rel, int64_t n, int64_t base) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (start2[i] < 0) start2[i] = base + rel[i];
}

// old rows (internal ids below nold): copied when they move (repack or
// outgrown slack), then the transposes of the new rows' entries appended;
// columns are stable internal ids, so rows that gain nothing are untouched
__global__ void k_move_old_rows(const int64_t* __restrict__ start_old, const int64_t* __restrict__ len_old,
                                int64_t nold, const int32_t* col_src, const double* val_src,
                                const int64_t* __restrict__ start2, int32_t* col_dst, double* val_dst,
                                const ulonglong2* __restrict__ T, const int64_t* __restrict__ tstart,
                                const int64_t* __restrict__ hist, const double* __restrict__ valN) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < nold; r += nwarps) {
    const int64_t src = start_old[r], dst = start2[r], len = len_old[r];
    const int64_t tn = hist[r];
    const bool moved = (dst != src) || (col_dst != col_src);
    if (!moved && tn == 0) continue;
    if (moved) {
      int64_t k = lane;
      for (; k + 96 < len; k += 128) {
        const int32_t j0 = col_src[src + k], j1 = col_src[src + k + 32], j2 = col_src[src + k + 64],
                      j3 = col_src[src + k + 96];
        const double v0 = val_src[src + k], v1 = val_src[src + k + 32], v2 = val_src[src + k + 64],
                     v3 = val_src[src + k + 96];
        col_dst[dst + k] = j0; col_dst[dst + k + 32] = j1; col_dst[dst + k + 64] = j2; col_dst[dst + k + 96] = j3;
        val_dst[dst + k] = v0; val_dst[dst + k + 32] = v1; val_dst[dst + k + 64] = v2; val_dst[dst + k + 96] = v3;
      }
      for (; k < len; k += 32) {
        col_dst[dst + k] = col_src[src + k];
        val_dst[dst + k] = val_src[src + k];
      }
    }
    const int64_t t0 = tstart[r];
    for (int64_t k = lane; k < tn; k += 32) {
      const ulonglong2 t = T[t0 + k];
      col_dst[dst + len + k] = (int32_t)(nold + (int64_t)(t.x >> 32));
      val_dst[dst + len + k] = valN[t.y];
    }
  }
}

__global__ void k_place_new_rows(int64_t nold, int64_t nnew, const int64_t* __restrict__ rpN,
                                 const int32_t* __restrict__ colN, const double* __restrict__ valN,
                                 const int64_t* __restrict__ start2, int32_t* __restrict__ col_dst,
                                 double* __restrict__ val_dst) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp; q < nnew; q += nwarps) {
    const int64_t dst = start2[nold + q];
    const int64_t b = rpN[q], len = rpN[q + 1] - b;
    for (int64_t k = lane; k < len; k += 32) {
      col_dst[dst + k] = colN[b + k];
      val_dst[dst + k] = valN[b + k];
    }
  }
}

// sorted <-> internal maps of V' and the keys in internal order
__global__ void k_build_perm(const int64_t* __restrict__ pos_old, const int32_t* __restrict__ s2i_old, int64_t nold,
                             const int32_t* __restrict__ newrows, int64_t nnew, const ulonglong2* __restrict__ V,
                             int32_t* __restrict__ s2i, int32_t* __restrict__ i2s, ulonglong2* __restrict__ keys_int) {
  const int64_t tot = nold + nnew;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < nold) {
      const int64_t p = pos_old[t];
      const int32_t id = s2i_old[t];
      s2i[p] = id;
      i2s[id] = (int32_t)p;
    } else {
      const int64_t q = t - nold;
      const int32_t p = newrows[q];
      const int64_t id = nold + q;
      s2i[p] = (int32_t)id;
      i2s[id] = p;
      keys_int[id] = V[p];
    }
  }
}

__global__ void k_iota(int32_t* __restrict__ a, int32_t* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = b[i] = (int32_t)i;
}

// out[t] = in[idx[t]] for nvec vectors of length n
__global__ void k_gather_vec(const double* __restrict__ in, const int32_t* __restrict__ idx, int64_t n, int nvec,
                             double* __restrict__ out) {
  const int64_t tot = n * nvec;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / n, i = t % n;
    out[t] = in[v * n + idx[i]];
  }
}


// diagonal <D|H|D> (includes e_core)
__global__ void k_diag(int n, const double* __restrict__ h, const double* __restrict__ eri, double ecore,
                       const ulonglong2* __restrict__ V, int64_t nV, double* __restrict__ out,
                       const int32_t* __restrict__ rowlist) {
  extern __shared__ double sm[];
  double* J = sm;            // (kk|ll)
  double* K = sm + n * n;    // (kl|lk)
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int k = t / n, l = t % n;
    J[t] = eri[(((int64_t)k * n + k) * n + l) * n + l];
    K[t] = eri[(((int64_t)k * n + l) * n + l) * n + k];
  }
  __syncthreads();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nV; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = rowlist ? (int64_t)rowlist[t] : t;
    ulonglong2 key = V[i];
    double e1 = 0.0, e2 = 0.0;
    for (int s = 0; s < 2; ++s) {
      uint64_t x = s == 0 ? key.x : key.y;
      uint64_t o = s == 0 ? key.y : key.x;
      uint64_t a = x;
      while (a) {
        int k = __ffsll((long long)a) - 1;
        a &= a - 1;
        e1 += h[k * n + k];
        // same spin pairs l > k, opposite spin pairs counted once (s == 0)
        uint64_t b = x & ~((2ull << k) - 1ull);
        while (b) {
          int l = __ffsll((long long)b) - 1;
          b &= b - 1;
          e2 += J[k * n + l] - K[k * n + l];
        }
        if (s == 0) {
          uint64_t c = o;
          while (c) {
            int l = __ffsll((long long)c) - 1;
            c &= c - 1;
            e2 += J[k * n + l];
          }
        }
      }
    }
    out[i] = ecore + e1 + e2;
  }
}

// Both-orientation form: sigma = diag .* c + offdiag * c ; one warp per row.  In the single-vector
// path each warp owns a contiguous range of rows holding an equal share of
// the connections and keeps four (col, val, c[col]) loads per lane in
// flight; the CSR stream is read with evict-first hints so that c stays in
// L2.  Rows are summed four at a time, so that the cross-lane reduction
// costs 1.5 FP64 additions per row instead of 8 (the FP64 pipe, 2 DFMA per
// clock per SM, bounds this kernel).
// blocks of k_sigma1 per SM, all resident (the grid is this many per SM)
constexpr int SIGMA_BLOCKS_PER_SM = 5;

__global__ void __launch_bounds__(256, SIGMA_BLOCKS_PER_SM) k_sigma1(const int64_t* __restrict__ rowptr,
                                                  const int64_t* __restrict__ rowstart, const int32_t* __restrict__ col,
                                               const double* __restrict__ val, const double* __restrict__ diag,
                                               int64_t nV, const double* __restrict__ c, double* __restrict__ sigma,
                                               int nvec_unused) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  {
    // contiguous row ranges holding an equal share of the connections
    const int64_t tot = rowptr[nV];
    const int64_t chunk = (tot + nwarps - 1) / nwarps;
    int64_t r0, r1;
    {
      int64_t lo = 0, hi = nV, x = warp * chunk;
      while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (rowptr[mid] < x) lo = mid + 1; else hi = mid; }
      r0 = lo;
      lo = r0; hi = nV; x = (warp + 1) * chunk;
      while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (rowptr[mid] < x) lo = mid + 1; else hi = mid; }
      r1 = warp == nwarps - 1 ? nV : lo;
    }
    for (int64_t g = r0; g < r1; g += 4) {
      double acc[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        double a = 0.0, a2 = 0.0;   // two chains, so consecutive FMAs do not wait on each other
        const int64_t i = g + r;
        if (i < r1) {
          const int64_t b = rowstart[i], e = b + (rowptr[i + 1] - rowptr[i]);
          int64_t k = b + lane;
          for (; k + 96 < e; k += 128) {
            const int32_t j0 = __ldcs(col + k), j1 = __ldcs(col + k + 32), j2 = __ldcs(col + k + 64),
                          j3 = __ldcs(col + k + 96);
            const double v0 = __ldcs(val + k), v1 = __ldcs(val + k + 32), v2 = __ldcs(val + k + 64),
                         v3 = __ldcs(val + k + 96);
            a = fma(v0, c[j0], a);
            a2 = fma(v1, c[j1], a2);
            a = fma(v2, c[j2], a);
            a2 = fma(v3, c[j3], a2);
          }
          for (; k < e; k += 32) a = fma(__ldcs(val + k), c[__ldcs(col + k)], a);
        }
        acc[r] = a + a2;
      }
      // four row sums at once: halve the values held per lane across lanes
      // 16 apart, then 8 apart, then a plain tree over the last 8 lanes
      const bool h16 = lane & 16, h8 = lane & 8;
      const double w0 = (h16 ? acc[2] : acc[0]) + __shfl_xor_sync(0xffffffffu, h16 ? acc[0] : acc[2], 16);
      const double w1 = (h16 ? acc[3] : acc[1]) + __shfl_xor_sync(0xffffffffu, h16 ? acc[1] : acc[3], 16);
      double u = (h8 ? w1 : w0) + __shfl_xor_sync(0xffffffffu, h8 ? w0 : w1, 8);
      u += __shfl_xor_sync(0xffffffffu, u, 4);
      u += __shfl_xor_sync(0xffffffffu, u, 2);
      u += __shfl_xor_sync(0xffffffffu, u, 1);
      if ((lane & 7) == 0) {
        const int64_t i = g + (h16 ? 2 : 0) + (h8 ? 1 : 0);
        if (i < r1) sigma[i] = fma(diag[i], c[i], u);
      }
    }
  }
}

// several vectors at once (one pass over the connections per 4 vectors)
__global__ void __launch_bounds__(256) k_sigma(const int64_t* __restrict__ rowptr,
                                               const int64_t* __restrict__ rowstart, const int32_t* __restrict__ col,
                                               const double* __restrict__ val, const double* __restrict__ diag,
                                               int64_t nV, const double* __restrict__ c, double* __restrict__ sigma,
                                               int nvec) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < nV; i += nwarps) {
    const int64_t b = rowstart[i], e = b + (rowptr[i + 1] - rowptr[i]);
    for (int v0 = 0; v0 < nvec; v0 += 4) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      const int nv = nvec - v0 < 4 ? nvec - v0 : 4;
      for (int64_t k = b + lane; k < e; k += 32) {
        const int64_t j = col[k];
        const double hv = val[k];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < nv) acc[t] = fma(hv, c[(int64_t)(v0 + t) * nV + j], acc[t]);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        double a = acc[t];
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        acc[t] = a;
      }
      if (lane < nv) {
        double a = lane == 0 ? acc[0] : lane == 1 ? acc[1] : lane == 2 ? acc[2] : acc[3];
        const int64_t o = (int64_t)(v0 + lane) * nV + i;
        sigma[o] = fma(diag[i], c[o], a);
      }
    }
  }
}

// The stored half of row i: its entries' columns and values.
__device__ __forceinline__ void row_entries(const SegTab& T, int64_t rs, const int32_t*& col, const double*& val) {
  const int sg = (int)(rs >> GRAPH_SEG_SHIFT);
  const int64_t o = rs & GRAPH_SEG_MASK;
  col = T.col[sg] + o;
  val = T.val[sg] + o;
}

// One-orientation form: sigma = diag .* c + H_off c.  Each stored entry (i, j, v), j < i, adds
// v c_j to sigma_i (the row sum) and v c_i to sigma_j (an FP64 atomic add
// into sigma, which stays in L2); sigma is zeroed before the launch and each
// row's sum is added atomically too, since other rows scatter into it at the
// same time.  One warp per contiguous range of rows holding an equal share
// of the entries, four (col, val, c[col]) loads per lane in flight, the entry
// stream read with evict-first hints so that c and sigma stay in L2.  Rows
// are summed four at a time, as in k_sigma1: the FP64 pipe (2 operations per
// entry, 2 DFMA per clock per SM) bounds this kernel (80% busy on the
// pentacene space), and stored rows are half as long as full ones.
// blocks of k_sigma1_half per SM: all resident (64 registers, no spills), so
// the equal shares of the entries run in one wave
constexpr int SIGMA_HALF_BLOCKS_PER_SM = 4;

// PASS 0: both contributions of every entry (sigma zeroed first).  When c
// and sigma do not fit L2 together, two passes keep one random-access
// vector in L2 each: PASS 1 writes sigma_i = H_ii c_i + the row sum (plain
// stores, no atomics, no zeroing), PASS 2 then adds the scatters.
template <int PASS>
__global__ void __launch_bounds__(256, SIGMA_HALF_BLOCKS_PER_SM) k_sigma1_half(const int64_t* __restrict__ rowptr,
                                                  const int64_t* __restrict__ rowstart, const __grid_constant__ SegTab T,
                                                  const double* __restrict__ diag, int64_t nV,
                                                  const double* __restrict__ c, double* sigma) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // contiguous row ranges holding an equal share of the entries
  const int64_t tot = rowptr[nV];
  const int64_t chunk = (tot + nwarps - 1) / nwarps;
  int64_t r0, r1;
  {
    int64_t lo = 0, hi = nV, x = warp * chunk;
    while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (rowptr[mid] < x) lo = mid + 1; else hi = mid; }
    r0 = lo;
    lo = r0; hi = nV; x = (warp + 1) * chunk;
    while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (rowptr[mid] < x) lo = mid + 1; else hi = mid; }
    r1 = warp == nwarps - 1 ? nV : lo;
  }
  for (int64_t g = r0; g < r1; g += 4) {
    double acc[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      double a = 0.0;
      const int64_t i = g + r;
      if (i < r1) {
        const int64_t len = rowptr[i + 1] - rowptr[i];
        const int32_t* col;
        const double* val;
        row_entries(T, rowstart[i], col, val);
        const double ci = c[i];
        int64_t k = lane;
        if (PASS != 2 || ci != 0.0) {
          for (; k + 96 < len; k += 128) {
            const int32_t j0 = __ldcs(col + k), j1 = __ldcs(col + k + 32), j2 = __ldcs(col + k + 64),
                          j3 = __ldcs(col + k + 96);
            const double v0 = __ldcs(val + k), v1 = __ldcs(val + k + 32), v2 = __ldcs(val + k + 64),
                         v3 = __ldcs(val + k + 96);
            if (PASS != 2) {
              a = fma(v0, c[j0], a);
              a = fma(v1, c[j1], a);
              a = fma(v2, c[j2], a);
              a = fma(v3, c[j3], a);
            }
            if (PASS != 1) {
              atomicAdd(sigma + j0, v0 * ci);
              atomicAdd(sigma + j1, v1 * ci);
              atomicAdd(sigma + j2, v2 * ci);
              atomicAdd(sigma + j3, v3 * ci);
            }
          }
          for (; k < len; k += 32) {
            const int32_t j = __ldcs(col + k);
            const double v = __ldcs(val + k);
            if (PASS != 2) a = fma(v, c[j], a);
            if (PASS != 1) atomicAdd(sigma + j, v * ci);
          }
        }
      }
      acc[r] = a;
    }
    // four row sums at once (1.5 FP64 additions per row for the cross-lane
    // reduction instead of 5): halve the values held per lane across lanes
    // 16 apart, then 8 apart, then a plain tree over the last 8 lanes
    const bool h16 = lane & 16, h8 = lane & 8;
    const double w0 = (h16 ? acc[2] : acc[0]) + __shfl_xor_sync(0xffffffffu, h16 ? acc[0] : acc[2], 16);
    const double w1 = (h16 ? acc[3] : acc[1]) + __shfl_xor_sync(0xffffffffu, h16 ? acc[1] : acc[3], 16);
    double u = (h8 ? w1 : w0) + __shfl_xor_sync(0xffffffffu, h8 ? w0 : w1, 8);
    u += __shfl_xor_sync(0xffffffffu, u, 4);
    u += __shfl_xor_sync(0xffffffffu, u, 2);
    u += __shfl_xor_sync(0xffffffffu, u, 1);
    if (PASS != 2 && (lane & 7) == 0) {
      const int64_t i = g + (h16 ? 2 : 0) + (h8 ? 1 : 0);
      if (i < r1) {
        if (PASS == 0) atomicAdd(sigma + i, fma(diag[i], c[i], u));
        else sigma[i] = fma(diag[i], c[i], u);
      }
    }
  }
}

// Rows r0 .. nV-1 of H c for a vector that vanishes on them (the rows a
// space gained in its last extension): out[i] = sum of the row's stored
// entries times c (both forms store every connection of such a row to an
// earlier determinant in the row itself); one warp per row.
__global__ void __launch_bounds__(256) k_sigma_tail(const int64_t* __restrict__ rowptr,
                                                    const int64_t* __restrict__ rowstart,
                                                    const __grid_constant__ SegTab T, int64_t r0, int64_t nV,
                                                    const double* __restrict__ c, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = r0 + warp; i < nV; i += nwarps) {
    const int64_t len = rowptr[i + 1] - rowptr[i];
    const int32_t* col;
    const double* val;
    row_entries(T, rowstart[i], col, val);
    double a = 0.0;
    for (int64_t k = lane; k < len; k += 32) a = fma(__ldcs(val + k), c[__ldcs(col + k)], a);
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) out[i] = a;
  }
}

// several vectors at once (one pass over the entries per 4 vectors); sigma
// zeroed before the launch, as for k_sigma1
__global__ void __launch_bounds__(256) k_sigma_half(const int64_t* __restrict__ rowptr,
                                               const int64_t* __restrict__ rowstart, const __grid_constant__ SegTab T,
                                               const double* __restrict__ diag, int64_t nV,
                                               const double* __restrict__ c, double* sigma, int nvec) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < nV; i += nwarps) {
    const int64_t len = rowptr[i + 1] - rowptr[i];
    const int32_t* col;
    const double* val;
    row_entries(T, rowstart[i], col, val);
    for (int v0 = 0; v0 < nvec; v0 += 4) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      double cin[4] = {0.0, 0.0, 0.0, 0.0};
      const int nv = nvec - v0 < 4 ? nvec - v0 : 4;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nv) cin[t] = c[(int64_t)(v0 + t) * nV + i];
      for (int64_t k = lane; k < len; k += 32) {
        const int64_t j = col[k];
        const double hv = val[k];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < nv) {
            acc[t] = fma(hv, c[(int64_t)(v0 + t) * nV + j], acc[t]);
            atomicAdd(sigma + (int64_t)(v0 + t) * nV + j, hv * cin[t]);
          }
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        double a = acc[t];
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        acc[t] = a;
      }
      if (lane < nv) {
        double a = lane == 0 ? acc[0] : lane == 1 ? acc[1] : lane == 2 ? acc[2] : acc[3];
        const int64_t o = (int64_t)(v0 + lane) * nV + i;
        atomicAdd(sigma + o, fma(diag[i], c[o], a));
      }
    }
  }
}

}  // namespace

// Group structures of the space in G.keys (nV determinants): alpha groups,
// beta-major order and beta groups, single-excitation neighbour lists of the
// distinct alpha and beta strings, and the (C) search cost per string.
static void space_args(hci_ctx* ctx, int64_t nV, GraphArgs& A);

static hci_status build_space(hci_ctx* ctx, int64_t nV, GraphArgs& A) {
  Graph& G = ctx->graph;
  prof_tic(ctx, HCI_PH_GRAPH_SPACE);
  const int n = ctx->n;
  const ulonglong2* V = bp<ulonglong2>(G.keys);
  int64_t* dtot = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 40);
  HCI_TRY(ensure_buf(ctx, ctx->s_flags, (size_t)(2 * nV + 1) * 8));
  int64_t* flag = bp<int64_t>(ctx->s_flags);
  int64_t* excl = flag + nV;
  HCI_TRY(ensure_buf(ctx, ctx->g_ia, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, ctx->g_ua, (size_t)nV * 8));
  HCI_TRY(ensure_buf(ctx, ctx->g_ga, (size_t)(nV + 1) * 8));
  const int gb = grid_for(nV, 256);
  HCI_LAUNCH(k_run_flags, gb, 256, 0, ctx->st)(V, nV, flag);
  HCI_TRY(scan_i64(ctx, flag, excl, nV, dtot));
  HCI_LAUNCH(k_groups, gb, 256, 0, ctx->st)(V, nV, flag, excl, bp<int32_t>(ctx->g_ia), bp<uint64_t>(ctx->g_ua),
                                             bp<int64_t>(ctx->g_ga));
  HCI_LAUNCH(k_set_last, 1, 1, 0, ctx->st)(bp<int64_t>(ctx->g_ga), dtot, nV);
  int64_t nua = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&nua, dtot, 8, cudaMemcpyDeviceToHost, ctx->st));
  HCI_TRY(ensure_buf(ctx, ctx->g_bkeys, (size_t)nV * 16));
  HCI_TRY(ensure_buf(ctx, ctx->g_bkeys2, (size_t)nV * 16));
  HCI_LAUNCH(k_swap_keys, gb, 256, 0, ctx->st)(V, nV, bp<ulonglong2>(ctx->g_bkeys));
  HCI_TRY(sort_keys(ctx, bp<uint64_t>(ctx->g_bkeys), bp<uint64_t>(ctx->g_bkeys2), nV, n, n));
  HCI_TRY(ensure_buf(ctx, ctx->g_ub, (size_t)nV * 8));
  HCI_TRY(ensure_buf(ctx, ctx->g_gb, (size_t)(nV + 1) * 8));
  HCI_TRY(ensure_buf(ctx, ctx->g_ib, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, ctx->g_permb, (size_t)nV * 4));
  int32_t* bgroup_of_pos = bp<int32_t>(ctx->g_bkeys2);
  HCI_LAUNCH(k_run_flags, gb, 256, 0, ctx->st)(bp<ulonglong2>(ctx->g_bkeys), nV, flag);
  HCI_TRY(scan_i64(ctx, flag, excl, nV, dtot));
  HCI_LAUNCH(k_groups, gb, 256, 0, ctx->st)(bp<ulonglong2>(ctx->g_bkeys), nV, flag, excl, bgroup_of_pos,
                                             bp<uint64_t>(ctx->g_ub), bp<int64_t>(ctx->g_gb));
  HCI_LAUNCH(k_set_last, 1, 1, 0, ctx->st)(bp<int64_t>(ctx->g_gb), dtot, nV);
  HCI_TRY(ensure_buf(ctx, ctx->g_posb, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, ctx->g_vb, (size_t)nV * 8));
  HCI_TRY(ensure_buf(ctx, ctx->g_ba, (size_t)nV * 8));
  HCI_LAUNCH(k_perm_b, gb, 256, 0, ctx->st)(bp<ulonglong2>(ctx->g_bkeys), nV, V, bgroup_of_pos,
                                             bp<int32_t>(ctx->g_permb), bp<int32_t>(ctx->g_ib),
                                             bp<int32_t>(ctx->g_posb), bp<uint64_t>(ctx->g_ba));
  HCI_LAUNCH(k_pack_beta, gb, 256, 0, ctx->st)(V, nV, bp<uint64_t>(ctx->g_vb));
  int64_t nub = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&nub, dtot, 8, cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaGetLastError());
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  G.nua = nua;
  G.nub = nub;
  // neighbour lists of both spins
  DevBuf* ptrs[2] = {&ctx->g_nbr_ptr, &ctx->g_bnbr_ptr};
  DevBuf* lists[2] = {&ctx->g_nbr, &ctx->g_bnbr};
  DevBuf* costs[2] = {&ctx->g_costa, &ctx->g_costb};
  const uint64_t* uniq[2] = {bp<uint64_t>(ctx->g_ua), bp<uint64_t>(ctx->g_ub)};
  const int64_t* gstart[2] = {bp<int64_t>(ctx->g_ga), bp<int64_t>(ctx->g_gb)};
  const int64_t nu[2] = {nua, nub};
  // lookups on the alpha side generate beta singles and vice versa
  const int Lside[2] = {ctx->nb * (n - ctx->nb), ctx->na * (n - ctx->na)};
  const int nel[2] = {ctx->na, ctx->nb};
  for (int s = 0; s < 2; ++s) {
    uint64_t tsize = 64;
    while (tsize < (uint64_t)(2 * nu[s] + 2)) tsize <<= 1;
    HCI_TRY(ensure_buf(ctx, ctx->g_htab, (size_t)tsize * 8));
    HCI_TRY(ensure_buf(ctx, ctx->g_hval, (size_t)tsize * 4));
    HCI_CUDA(ctx, cudaMemsetAsync(ctx->g_htab.p, 0xFF, (size_t)tsize * 8, ctx->st));
    HCI_LAUNCH(k_hash_insert, grid_for(nu[s], 256), 256, 0, ctx->st)(uniq[s], nu[s], bp<unsigned long long>(ctx->g_htab),
                                                                      bp<int32_t>(ctx->g_hval), tsize - 1);
    HCI_TRY(ensure_buf(ctx, ctx->g_cnt, (size_t)(nu[s] + 1) * 8));
    HCI_TRY(ensure_buf(ctx, *ptrs[s], (size_t)(nu[s] + 1) * 8));
    HCI_TRY(ensure_buf(ctx, *costs[s], (size_t)(nu[s] + 1) * 8));
    const int gw = grid_for(nu[s] * 32, 256);
    // one pass of hash look-ups when the padded lists (every string's
    // largest possible list) take at most 1 GB, else a count pass and a
    // fill pass
    const int Lown = nel[s] * (n - nel[s]);
    const size_t scr_bytes = (size_t)nu[s] * (size_t)(Lown > 0 ? Lown : 1) * 4;
    const bool one_pass = scr_bytes <= ((size_t)1 << 30);
    if (one_pass) HCI_TRY(ensure_buf(ctx, ctx->g_nscr, scr_bytes));
    HCI_LAUNCH(k_alpha_nbrs, gw, 256, 0, ctx->st)(n, nel[s], uniq[s], nu[s], nullptr, bp<int64_t>(ctx->g_cnt), nullptr,
                                                   bp<unsigned long long>(ctx->g_htab), bp<int32_t>(ctx->g_hval),
                                                   tsize - 1, one_pass ? bp<int32_t>(ctx->g_nscr) : nullptr);
    HCI_TRY(scan_i64(ctx, bp<int64_t>(ctx->g_cnt), bp<int64_t>(*ptrs[s]), nu[s], dtot));
    HCI_LAUNCH(k_store_at, 1, 1, 0, ctx->st)(bp<int64_t>(*ptrs[s]), nu[s], dtot);
    int64_t nn = 0;
    HCI_CUDA(ctx, cudaMemcpyAsync(&nn, dtot, 8, cudaMemcpyDeviceToHost, ctx->st));
    HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
    HCI_TRY(ensure_buf(ctx, *lists[s], (size_t)(nn + 1) * 4));
    if (one_pass)
      HCI_LAUNCH(k_compact_nbrs, gw, 256, 0, ctx->st)(bp<int32_t>(ctx->g_nscr), Lown, bp<int64_t>(*ptrs[s]), nu[s],
                                                       bp<int32_t>(*lists[s]));
    else
      HCI_LAUNCH(k_alpha_nbrs, gw, 256, 0, ctx->st)(n, nel[s], uniq[s], nu[s], bp<int64_t>(*ptrs[s]), nullptr,
                                                     bp<int32_t>(*lists[s]), bp<unsigned long long>(ctx->g_htab),
                                                     bp<int32_t>(ctx->g_hval), tsize - 1, nullptr);
    HCI_LAUNCH(k_nbr_cost, gw, 256, 0, ctx->st)(bp<int64_t>(*ptrs[s]), bp<int32_t>(*lists[s]), gstart[s], nu[s],
                                                 Lside[s], bp<int64_t>(*costs[s]));
  }
  HCI_CUDA(ctx, cudaGetLastError());
  space_args(ctx, nV, A);
  prof_toc(ctx, HCI_PH_GRAPH_SPACE);
  return HCI_OK;
}

// Traversal arguments of the space built by build_space (pointers only).
static void space_args(hci_ctx* ctx, int64_t nV, GraphArgs& A) {
  const int n = ctx->n;
  A = GraphArgs{};
  A.V = bp<ulonglong2>(ctx->graph.keys);
  A.bk = bp<ulonglong2>(ctx->g_bkeys);
  A.nV = nV;
  A.n = n; A.na = ctx->na; A.nb = ctx->nb;
  A.ia = bp<int32_t>(ctx->g_ia); A.ga = bp<int64_t>(ctx->g_ga);
  A.ib = bp<int32_t>(ctx->g_ib); A.gb = bp<int64_t>(ctx->g_gb);
  A.permb = bp<int32_t>(ctx->g_permb);
  A.vb = bp<uint64_t>(ctx->g_vb);
  A.ba = bp<uint64_t>(ctx->g_ba);
  A.posb = bp<int32_t>(ctx->g_posb);
  A.anbr_ptr = bp<int64_t>(ctx->g_nbr_ptr); A.anbr = bp<int32_t>(ctx->g_nbr);
  A.bnbr_ptr = bp<int64_t>(ctx->g_bnbr_ptr); A.bnbr = bp<int32_t>(ctx->g_bnbr);
  A.costa = bp<int64_t>(ctx->g_costa); A.costb = bp<int64_t>(ctx->g_costb);
  A.H = HamView{n,
                bp<double>(ctx->h),
                bp<double>(ctx->eri),
                bp<double>(ctx->jk_same),
                bp<double>(ctx->j_opp),
                bp<double>(ctx->lists.f_ref),
                ctx->na == 64 ? ~0ull : ((1ull << ctx->na) - 1ull),
                ctx->nb == 64 ? ~0ull : ((1ull << ctx->nb) - 1ull)};
  A.queue = reinterpret_cast<unsigned long long*>(bp<char>(ctx->s_counter) + 48);
  A.rowlist = nullptr;
  A.nrows = nV;
  A.rowptr = nullptr; A.col = nullptr; A.val = nullptr; A.rowcnt = nullptr;
  A.scr = nullptr; A.scr_cap = 0; A.stage = nullptr; A.stage_cap = 0; A.rowoff = nullptr; A.stage_ctl = nullptr;
  A.s2i = bp<int32_t>(ctx->graph.s2i);
  A.lower = 0;
  A.dc = nullptr; A.dsig = nullptr; A.ddiag = nullptr; A.dnnz = nullptr;
}

// Count the entries of the rows listed in A (A.rowlist / A.nrows) into cnt.
static hci_status rows_count(hci_ctx* ctx, GraphArgs& A, DevBuf& cnt) {
  HCI_TRY(ensure_buf(ctx, cnt, (size_t)(A.nrows + 1) * 8));
  A.rowcnt = bp<int64_t>(cnt);
  A.rowptr = nullptr; A.col = nullptr; A.val = nullptr;
  HCI_CUDA(ctx, cudaMemsetAsync(A.queue, 0, 8, ctx->st));
  HCI_LAUNCH(k_rows<ROWS_COUNT>, rows_grid(ctx), G_WARPS * 32, 0, ctx->st)(A);
  HCI_CUDA(ctx, cudaGetLastError());
  A.rowcnt = nullptr;
  return HCI_OK;
}

// Fill the listed rows, row q starting at offs[q] of col/val.
static hci_status rows_fill(hci_ctx* ctx, GraphArgs& A, const int64_t* offs, int32_t* col, double* val) {
  A.rowptr = offs; A.col = col; A.val = val;
  HCI_CUDA(ctx, cudaMemsetAsync(A.queue, 0, 8, ctx->st));
  HCI_LAUNCH(k_rows<ROWS_FILL>, rows_grid(ctx), G_WARPS * 32, 0, ctx->st)(A);
  HCI_CUDA(ctx, cudaGetLastError());
  return HCI_OK;
}


static int64_t read_i64(hci_ctx* ctx, const int64_t* d, hci_status* st) {
  int64_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, d, 8, cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  *st = e == cudaSuccess ? HCI_OK : hci_fail(ctx, HCI_ERR_CUDA, "graph: %s", cudaGetErrorString(e));
  return v;
}

// The rows listed in A (rowlist, nrows; a list is required) searched once
// into per-warp scratch and a staging buffer (sized from est entries):
// counts into inc.cnt, their prefix sums into inc.rpN (inc.rpN[nrows] =
// *total), rows that outgrew the scratch or the staging space marked for a
// second search (*left of them).
static hci_status stage_search(hci_ctx* ctx, GraphArgs& A, int64_t est, int64_t* total, int64_t* left) {
  IncScratch& S = ctx->inc;
  cudaStream_t st = ctx->st;
  const int64_t nrows = A.nrows;
  int64_t* dtot = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 40);
  HCI_TRY(ensure_buf(ctx, S.cnt, (size_t)(nrows + 1) * 8));
  HCI_TRY(ensure_buf(ctx, S.roff, (size_t)(nrows + 1) * 8));
  HCI_TRY(ensure_buf(ctx, S.scr, (size_t)rows_grid(ctx) * G_WARPS * ROW_SCR * 4));
  if (S.stage.bytes < (size_t)est * 4) HCI_TRY(ensure_buf(ctx, S.stage, (size_t)est * 4));
  HCI_TRY(ensure_buf(ctx, S.ctl, 32));
  HCI_CUDA(ctx, cudaMemsetAsync(S.ctl.p, 0, 32, st));
  unsigned long long* ctl = bp<unsigned long long>(S.ctl);
  A.rowcnt = bp<int64_t>(S.cnt);
  A.scr = bp<int32_t>(S.scr);
  A.scr_cap = ROW_SCR;
  A.stage = bp<int32_t>(S.stage);
  A.stage_cap = (int64_t)(S.stage.bytes / 4);
  A.rowoff = bp<int64_t>(S.roff);
  A.stage_ctl = ctl;
  HCI_CUDA(ctx, cudaMemsetAsync(A.queue, 0, 8, st));
  HCI_LAUNCH(k_rows<ROWS_STAGED>, rows_grid(ctx), G_WARPS * 32, 0, st)(A);
  HCI_CUDA(ctx, cudaGetLastError());
  A.rowcnt = nullptr; A.scr = nullptr; A.scr_cap = 0; A.stage = nullptr; A.stage_cap = 0; A.rowoff = nullptr;
  A.stage_ctl = nullptr;
  HCI_TRY(ensure_buf(ctx, S.rpN, (size_t)(nrows + 1) * 8));
  HCI_TRY(scan_i64(ctx, bp<int64_t>(S.cnt), bp<int64_t>(S.rpN), nrows, dtot));
  HCI_LAUNCH(k_store_at, 1, 1, 0, st)(bp<int64_t>(S.rpN), nrows, dtot);
  hci_status hs = HCI_OK;
  *total = read_i64(ctx, dtot, &hs);
  HCI_TRY(hs);
  *left = read_i64(ctx, reinterpret_cast<const int64_t*>(ctl + 1), &hs);
  HCI_TRY(hs);
  return HCI_OK;
}

// Columns of the rows of stage_search written to col, row q at off[q]
// (default inc.rpN[q]; lens[q] entries, default the dense rpN differences):
// staged rows copied, the rows left searched again at their offsets (left <
// 0: no row was staged, all are searched again).
static hci_status stage_place(hci_ctx* ctx, GraphArgs& A, int64_t left, int32_t* col, const int64_t* off = nullptr,
                              const int64_t* lens = nullptr) {
  IncScratch& S = ctx->inc;
  cudaStream_t st = ctx->st;
  const int64_t nrows = A.nrows;
  if (!off) off = bp<int64_t>(S.rpN);
  if (left < 0) return rows_fill(ctx, A, off, col, nullptr);   // counted, not staged
  HCI_LAUNCH(k_copy_staged, grid_for(nrows * 32, 256), 256, 0, st)(bp<int64_t>(S.roff), off, lens, nrows,
                                                                    bp<int32_t>(S.stage), col);
  HCI_CUDA(ctx, cudaGetLastError());
  ctx->st_counts[HCI_ST_ROWS_REFILLED] += left;
  if (left > 0) {
    unsigned long long* ctl = bp<unsigned long long>(S.ctl);
    HCI_TRY(ensure_buf(ctx, S.left, (size_t)left * 12 + 16));
    int64_t* left_off = bp<int64_t>(S.left);
    int32_t* left_rows = reinterpret_cast<int32_t*>(left_off + left);
    HCI_LAUNCH(k_collect_left, grid_for(nrows, 256), 256, 0, st)(bp<int64_t>(S.roff), off, A.rowlist, nrows, ctl + 2,
                                                                  left_rows, left_off);
    const int32_t* rl = A.rowlist;
    A.rowlist = left_rows;
    A.nrows = left;
    hci_status fs = rows_fill(ctx, A, left_off, col, nullptr);
    A.rowlist = rl;
    A.nrows = nrows;
    HCI_TRY(fs);
  }
  return HCI_OK;
}

static hci_status compute_diag(hci_ctx* ctx, int64_t nrows, const ulonglong2* keys, double* out) {
  const int n = ctx->n;
  prof_tic(ctx, HCI_PH_HDIAG);
  HCI_CUDA(ctx, cudaFuncSetAttribute(k_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 8));
  if (nrows > 0)
    HCI_LAUNCH(k_diag, grid_for(nrows, 128), 128, (size_t)2 * n * n * 8, ctx->st)(
        n, bp<double>(ctx->h), bp<double>(ctx->eri), ctx->ecore, keys, nrows, out, nullptr);
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_HDIAG);
  return HCI_OK;
}

// b grown to at least `bytes` (a quarter more, for later growth), its first
// `keep` bytes preserved
static hci_status grow_keep(hci_ctx* ctx, DevBuf& b, size_t bytes, size_t keep) {
  if (b.p && b.bytes >= bytes) return HCI_OK;
  DevBuf& t = ctx->inc.grow;
  HCI_TRY(ensure_buf(ctx, t, bytes + bytes / 4));
  if (keep > 0 && b.p) HCI_CUDA(ctx, cudaMemcpyAsync(t.p, b.p, keep, cudaMemcpyDeviceToDevice, ctx->st));
  std::swap(b, t);
  free_buf(ctx->st, t);
  return HCI_OK;
}

static void free_segments(hci_ctx* ctx) {
  Graph& G = ctx->graph;
  for (int k = 0; k < GRAPH_MAXSEG; ++k) {
    free_buf(ctx->st, G.seg_col[k]);
    free_buf(ctx->st, G.seg_val[k]);
  }
  G.nseg = 0;
  G.nstored = 0;
  G.nnz = 0;
  G.pool_used = G.pool_cap = 0;
}

// A new segment of `entries` stored connections; HCI_ERR_NOMEM when the
// stored connections would exceed the context's budget.
static hci_status seg_alloc(hci_ctx* ctx, int64_t entries, int* seg) {
  Graph& G = ctx->graph;
  if (G.nseg >= GRAPH_MAXSEG) return hci_fail(ctx, HCI_ERR_INVALID, "graph: segment table full");
  const int64_t bytes = (G.nstored + entries) * 12;
  if (ctx->graph_budget > 0 && bytes > ctx->graph_budget)
    return hci_fail(ctx, HCI_ERR_NOMEM, "graph: %lld bytes of stored connections exceed the budget of %lld",
                    (long long)bytes, (long long)ctx->graph_budget);
  HCI_TRY(ensure_buf(ctx, G.seg_col[G.nseg], (size_t)(entries + 1) * 4));
  HCI_TRY(ensure_buf(ctx, G.seg_val[G.nseg], (size_t)(entries + 1) * 8));
  *seg = G.nseg++;
  return HCI_OK;
}

// The new rows listed in A searched once (stage_search), the staging space
// sized from the mean length of a strided sample of them (the old rows'
// lengths say little when the space grows many-fold).  When that space would
// exceed an eighth of device memory the rows are only counted here (*left =
// -1) and stage_place searches them a second time, straight into place.
static hci_status stage_new_rows(hci_ctx* ctx, GraphArgs& A, int64_t nnew, int64_t nV, int64_t* total, int64_t* left) {
  IncScratch& S = ctx->inc;
  cudaStream_t st = ctx->st;
  const int64_t ns = std::min<int64_t>(nnew, ROW_SAMPLE);
  HCI_TRY(ensure_buf(ctx, S.samp, (size_t)ns * 12 + 16));
  int64_t* samp_cnt = bp<int64_t>(S.samp);
  int32_t* samp_rows = reinterpret_cast<int32_t*>(samp_cnt + ns);
  HCI_LAUNCH(k_stride_sample, grid_for(ns, 256), 256, 0, st)(A.rowlist, nnew, ns, samp_rows);
  GraphArgs B = A;
  B.rowlist = samp_rows;
  B.nrows = ns;
  B.rowcnt = samp_cnt;
  HCI_CUDA(ctx, cudaMemsetAsync(B.queue, 0, 8, st));
  HCI_LAUNCH(k_rows<ROWS_COUNT>, rows_grid(ctx), G_WARPS * 32, 0, st)(B);
  HCI_CUDA(ctx, cudaGetLastError());
  std::vector<int64_t> cnt((size_t)ns);
  HCI_CUDA(ctx, cudaMemcpyAsync(cnt.data(), samp_cnt, (size_t)ns * 8, cudaMemcpyDeviceToHost, st));
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  double sum = 0.0;
  for (int64_t v : cnt) sum += (double)v;
  const double mean = ns > 0 ? sum / (double)ns : 0.0;
  const double want = 1.5 * (double)nnew * mean;
  const int64_t est = (int64_t)std::min((double)nnew * (double)nV, want) + ((int64_t)1 << 22);
  {
    // a graph that cannot fit device memory is refused before the search:
    // both orientations add the new rows, their transposes and slack to the
    // pool, one orientation adds the new rows
    const Graph& G = ctx->graph;
    const double rows = (double)nnew * mean;
    const double need = G.half ? (double)G.nstored + rows : (double)G.pool_used + 2.5 * rows;
    if (need * 12.0 > 0.9 * (double)ctx->mem_total)
      return hci_fail(ctx, HCI_ERR_NOMEM, "graph: about %.3g bytes of stored connections would exceed device memory",
                      need * 12.0);
  }
  if ((double)est * 4.0 > (double)ctx->mem_total / 8.0) {
    // a staging buffer this large would crowd out the stored rows: count
    // the rows first and let stage_place search them again into place
    int64_t* dtot = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 40);
    HCI_TRY(rows_count(ctx, A, S.cnt));
    HCI_TRY(ensure_buf(ctx, S.rpN, (size_t)(nnew + 1) * 8));
    HCI_TRY(scan_i64(ctx, bp<int64_t>(S.cnt), bp<int64_t>(S.rpN), nnew, dtot));
    HCI_LAUNCH(k_store_at, 1, 1, 0, st)(bp<int64_t>(S.rpN), nnew, dtot);
    hci_status hs = HCI_OK;
    *total = read_i64(ctx, dtot, &hs);
    *left = -1;
    return hs;
  }
  return stage_search(ctx, A, est, total, left);
}

static hci_status graph_build_half(hci_ctx* ctx, const uint64_t* keys, int64_t nV) {
  Graph& G = ctx->graph;
  G.valid = false;
  if (nV >= ((int64_t)1 << 31) - 1) return hci_fail(ctx, HCI_ERR_INVALID, "graph: nV exceeds int32 columns");
  free_segments(ctx);
  G.half = true;
  prof_tic(ctx, HCI_PH_GRAPH);
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  int64_t* dtot = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 40);
  HCI_TRY(ensure_buf(ctx, G.keys, (size_t)nV * 16));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.keys.p, keys, (size_t)nV * 16, cudaMemcpyDeviceToDevice, ctx->st));
  // a fresh space: internal ids = sorted positions
  HCI_TRY(ensure_buf(ctx, G.keys_int, (size_t)nV * 16));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.keys_int.p, keys, (size_t)nV * 16, cudaMemcpyDeviceToDevice, ctx->st));
  HCI_TRY(ensure_buf(ctx, G.s2i, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, G.i2s, (size_t)nV * 4));
  HCI_LAUNCH(k_iota, grid_for(nV, 256), 256, 0, ctx->st)(bp<int32_t>(G.s2i), bp<int32_t>(G.i2s), nV);
  GraphArgs A;
  HCI_TRY(build_space(ctx, nV, A));
  A.s2i = bp<int32_t>(G.s2i);
  A.lower = 1;
  prof_tic(ctx, HCI_PH_GRAPH_ROWS);
  // stored halves of the rows, each searched once (staged; the row list is
  // the identity map), into one segment, then their elements
  A.rowlist = bp<int32_t>(G.s2i);
  A.nrows = nV;
  int64_t nst = 0, left = 0;
  HCI_TRY(stage_new_rows(ctx, A, nV, nV, &nst, &left));
  HCI_TRY(ensure_buf(ctx, G.rowptr, (size_t)(nV + 1) * 8));
  HCI_TRY(ensure_buf(ctx, G.rowstart, (size_t)(nV + 1) * 8));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.rowptr.p, ctx->inc.rpN.p, (size_t)(nV + 1) * 8, cudaMemcpyDeviceToDevice, ctx->st));
  int seg = 0;
  HCI_TRY(seg_alloc(ctx, nst, &seg));
  int32_t* col = bp<int32_t>(G.seg_col[seg]);
  double* val = bp<double>(G.seg_val[seg]);
  HCI_TRY(stage_place(ctx, A, left, col));
  A.rowlist = nullptr;
  HCI_LAUNCH(k_row_values<true>, grid_for(nV * 32, 256), 256, 0, ctx->st)(
      nullptr, nV, bp<int64_t>(G.rowptr), nullptr, col, val, bp<ulonglong2>(G.keys), bp<ulonglong2>(G.keys_int), A.H);
  HCI_LAUNCH(k_append_rows, grid_for(nV + 1, 256), 256, 0, ctx->st)(0, nV, bp<int64_t>(G.rowptr), 0, seg,
                                                                     bp<int64_t>(G.rowptr), bp<int64_t>(G.rowstart));
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_GRAPH_ROWS);
  HCI_TRY(ensure_buf(ctx, G.diag, (size_t)nV * 8));
  HCI_TRY(compute_diag(ctx, nV, bp<ulonglong2>(G.keys_int), bp<double>(G.diag)));
  prof_toc(ctx, HCI_PH_GRAPH);
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  G.nV = nV;
  G.nstored = nst;
  G.nnz = 2 * nst;
  G.epoch += 1;
  G.parent = -1;
  ctx->st_counts[HCI_ST_GRAPH_BUILDS] += 1;
  G.valid = true;
  return HCI_OK;
}

// V' contains every determinant of the cached space.  Rows and columns of the
// graph are internal ids (insertion order): old determinants keep theirs and
// the new ones are numbered after them, so a connection between an old and a
// new determinant belongs to the new row, and the stored rows never change.
// Only the new rows are searched (once, staged), into one new segment.
static hci_status graph_extend_half(hci_ctx* ctx, const uint64_t* keys, int64_t nV, bool* done) {
  Graph& G = ctx->graph;
  IncScratch& S = ctx->inc;
  *done = false;
  const int64_t nold = G.nV;
  if (nV <= nold || nV >= ((int64_t)1 << 31) - 1 || G.nseg >= GRAPH_MAXSEG) return HCI_OK;
  cudaStream_t st = ctx->st;
  unsigned long long* missing = reinterpret_cast<unsigned long long*>(bp<char>(ctx->s_counter) + 24);
  int64_t* dtot = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 40);
  const ulonglong2* Vn = reinterpret_cast<const ulonglong2*>(keys);
  HCI_TRY(ensure_buf(ctx, S.pos_old, (size_t)nold * 8));
  HCI_TRY(ensure_buf(ctx, S.mark, (size_t)nV * 8));
  HCI_CUDA(ctx, cudaMemsetAsync(S.mark.p, 0, (size_t)nV * 8, st));
  HCI_CUDA(ctx, cudaMemsetAsync(missing, 0, 8, st));
  HCI_LAUNCH(k_find_old, grid_for(nold, 256), 256, 0, st)(bp<ulonglong2>(G.keys), nold, Vn, nV,
                                                          bp<int64_t>(S.pos_old), bp<int64_t>(S.mark), missing);
  unsigned long long miss = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&miss, missing, 8, cudaMemcpyDeviceToHost, st));
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  if (miss) return HCI_OK;        // not an extension: full rebuild
  prof_tic(ctx, HCI_PH_GRAPH);
  hci_status hs = HCI_OK;
  const int64_t nnew = nV - nold;
  // keys and map of the old space move to the scratch side
  std::swap(G.keys, S.keys_old);
  std::swap(G.s2i, S.s2i_old);
  HCI_TRY(ensure_buf(ctx, G.keys, (size_t)nV * 16));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.keys.p, keys, (size_t)nV * 16, cudaMemcpyDeviceToDevice, st));
  // new determinants in sorted order, their internal ids nold + q
  HCI_TRY(ensure_buf(ctx, S.flag, (size_t)(2 * nV + 1) * 8));
  int64_t* nflag = bp<int64_t>(S.flag);
  int64_t* npos = nflag + nV;
  HCI_LAUNCH(k_not, grid_for(nV, 256), 256, 0, st)(bp<int64_t>(S.mark), nV, nflag);
  HCI_TRY(scan_i64(ctx, nflag, npos, nV, dtot));
  HCI_TRY(ensure_buf(ctx, S.newrows, (size_t)nnew * 4));
  HCI_LAUNCH(k_compact_idx, grid_for(nV, 256), 256, 0, st)(nflag, npos, nV, bp<int32_t>(S.newrows));
  // maps and internal-order keys of V' (old ids and keys unchanged)
  HCI_TRY(ensure_buf(ctx, G.s2i, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, G.i2s, (size_t)nV * 4));
  HCI_TRY(grow_keep(ctx, G.keys_int, (size_t)nV * 16, (size_t)nold * 16));
  HCI_LAUNCH(k_build_perm, grid_for(nV, 256), 256, 0, st)(bp<int64_t>(S.pos_old), bp<int32_t>(S.s2i_old), nold,
                                                          bp<int32_t>(S.newrows), nnew, Vn, bp<int32_t>(G.s2i),
                                                          bp<int32_t>(G.i2s), bp<ulonglong2>(G.keys_int));
  GraphArgs A;
  HCI_TRY(build_space(ctx, nV, A));
  A.s2i = bp<int32_t>(G.s2i);
  A.lower = 1;
  A.rowlist = bp<int32_t>(S.newrows);
  A.nrows = nnew;
  prof_tic(ctx, HCI_PH_GRAPH_ROWS);
  int64_t total = 0, left = 0;
  HCI_TRY(stage_new_rows(ctx, A, nnew, nV, &total, &left));
  int seg = 0;
  HCI_TRY(seg_alloc(ctx, total, &seg));
  int32_t* col = bp<int32_t>(G.seg_col[seg]);
  double* val = bp<double>(G.seg_val[seg]);
  HCI_TRY(stage_place(ctx, A, left, col));
  HCI_LAUNCH(k_row_values<true>, grid_for(nnew * 32, 256), 256, 0, st)(
      bp<int32_t>(S.newrows), nnew, bp<int64_t>(S.rpN), nullptr, col, val, bp<ulonglong2>(G.keys),
      bp<ulonglong2>(G.keys_int), A.H);
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_GRAPH_ROWS);
  // row table: the new rows after the old ones
  prof_tic(ctx, HCI_PH_GRAPH_MERGE);
  HCI_TRY(grow_keep(ctx, G.rowptr, (size_t)(nV + 1) * 8, (size_t)(nold + 1) * 8));
  HCI_TRY(grow_keep(ctx, G.rowstart, (size_t)(nV + 1) * 8, (size_t)nold * 8));
  HCI_LAUNCH(k_append_rows, grid_for(nnew + 1, 256), 256, 0, st)(nold, nnew, bp<int64_t>(S.rpN), G.nstored, seg,
                                                                  bp<int64_t>(G.rowptr), bp<int64_t>(G.rowstart));
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_GRAPH_MERGE);
  // diagonal: old entries stay, the new ids are computed
  HCI_TRY(grow_keep(ctx, G.diag, (size_t)nV * 8, (size_t)nold * 8));
  HCI_TRY(compute_diag(ctx, nnew, bp<ulonglong2>(G.keys_int) + nold, bp<double>(G.diag) + nold));
  prof_toc(ctx, HCI_PH_GRAPH);
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  (void)hs;
  G.parent = G.epoch;
  G.epoch += 1;
  G.nold = nold;
  G.tail_entries = total;
  G.nV = nV;
  G.nstored += total;
  G.nnz = 2 * G.nstored;
  ctx->st_counts[HCI_ST_GRAPH_BUILDS] += 1;
  *done = true;
  return HCI_OK;
}

// entries the both-orientation pool (segment 0) holds
static int64_t pool_entries(const Graph& G) {
  const int64_t a = (int64_t)(G.seg_col[0].bytes / 4), b = (int64_t)(G.seg_val[0].bytes / 8);
  return a < b ? a : b;
}

static hci_status graph_build_full(hci_ctx* ctx, const uint64_t* keys, int64_t nV) {
  Graph& G = ctx->graph;
  G.valid = false;
  if (nV >= ((int64_t)1 << 31) - 1) return hci_fail(ctx, HCI_ERR_INVALID, "graph: nV exceeds int32 columns");
  free_segments(ctx);
  G.half = false;
  prof_tic(ctx, HCI_PH_GRAPH);
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  int64_t* dtot = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 40);
  HCI_TRY(ensure_buf(ctx, G.keys, (size_t)nV * 16));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.keys.p, keys, (size_t)nV * 16, cudaMemcpyDeviceToDevice, ctx->st));
  // a fresh space: internal ids = sorted positions
  HCI_TRY(ensure_buf(ctx, G.keys_int, (size_t)nV * 16));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.keys_int.p, keys, (size_t)nV * 16, cudaMemcpyDeviceToDevice, ctx->st));
  HCI_TRY(ensure_buf(ctx, G.s2i, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, G.i2s, (size_t)nV * 4));
  HCI_LAUNCH(k_iota, grid_for(nV, 256), 256, 0, ctx->st)(bp<int32_t>(G.s2i), bp<int32_t>(G.i2s), nV);
  GraphArgs A;
  HCI_TRY(build_space(ctx, nV, A));
  A.s2i = bp<int32_t>(G.s2i);
  prof_tic(ctx, HCI_PH_GRAPH_ROWS);
  // every row searched once (staged, as for the new rows of an extension;
  // the row list is the identity map), lengths and logical offsets from it
  A.rowlist = bp<int32_t>(G.s2i);
  A.nrows = nV;
  int64_t nnz = 0, left = 0;
  HCI_TRY(stage_new_rows(ctx, A, nV, nV, &nnz, &left));
  HCI_TRY(ensure_buf(ctx, G.rowlen, (size_t)(nV + 1) * 8));
  HCI_TRY(ensure_buf(ctx, G.rowptr, (size_t)(nV + 1) * 8));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.rowlen.p, ctx->inc.cnt.p, (size_t)nV * 8, cudaMemcpyDeviceToDevice, ctx->st));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.rowptr.p, ctx->inc.rpN.p, (size_t)(nV + 1) * 8, cudaMemcpyDeviceToDevice, ctx->st));
  // capacities with slack, starts = their prefix sums, pool with headroom
  HCI_TRY(ensure_buf(ctx, G.rowcap, (size_t)(nV + 1) * 8));
  HCI_TRY(ensure_buf(ctx, G.rowstart, (size_t)(nV + 1) * 8));
  HCI_LAUNCH(k_caps, grid_for(nV, 256), 256, 0, ctx->st)(bp<int64_t>(G.rowlen), nV, bp<int64_t>(G.rowcap));
  HCI_TRY(scan_i64(ctx, bp<int64_t>(G.rowcap), bp<int64_t>(G.rowstart), nV, dtot));
  hci_status st = HCI_OK;
  const int64_t used = read_i64(ctx, dtot, &st);
  HCI_TRY(st);
  const int64_t cap = used + used / 4 + 1024;
  if (ctx->graph_budget > 0 && cap * 12 > ctx->graph_budget)
    return hci_fail(ctx, HCI_ERR_NOMEM, "graph: a pool of %lld bytes exceeds the budget of %lld", (long long)(cap * 12),
                    (long long)ctx->graph_budget);
  HCI_TRY(ensure_buf(ctx, G.seg_col[0], (size_t)cap * 4));
  HCI_TRY(ensure_buf(ctx, G.seg_val[0], (size_t)cap * 8));
  G.nseg = 1;
  HCI_TRY(stage_place(ctx, A, left, bp<int32_t>(G.seg_col[0]), bp<int64_t>(G.rowstart), bp<int64_t>(G.rowlen)));
  A.rowlist = nullptr;
  HCI_LAUNCH(k_row_values<false>, grid_for(nV * 32, 256), 256, 0, ctx->st)(
      nullptr, nV, bp<int64_t>(G.rowstart), bp<int64_t>(G.rowlen), bp<int32_t>(G.seg_col[0]),
      bp<double>(G.seg_val[0]), bp<ulonglong2>(G.keys), bp<ulonglong2>(G.keys_int), A.H);
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_GRAPH_ROWS);
  HCI_TRY(ensure_buf(ctx, G.diag, (size_t)nV * 8));
  HCI_TRY(compute_diag(ctx, nV, bp<ulonglong2>(G.keys_int), bp<double>(G.diag)));
  prof_toc(ctx, HCI_PH_GRAPH);
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  G.nV = nV;
  G.nnz = nnz;
  G.nstored = nnz;
  G.epoch += 1;
  G.parent = -1;
  G.pool_used = used;
  G.pool_cap = pool_entries(G);
  ctx->st_counts[HCI_ST_GRAPH_BUILDS] += 1;
  G.valid = true;
  return HCI_OK;
}

// V' contains every determinant of the cached space.  Rows and columns of the
// graph are internal ids (insertion order): old determinants keep theirs and
// the new ones are numbered after them, so only the new rows are searched,
// their transposes are appended to the old rows (in place where the row's
// slack allows), and no stored column changes.
static hci_status graph_extend_full(hci_ctx* ctx, const uint64_t* keys, int64_t nV, bool* done) {
  Graph& G = ctx->graph;
  IncScratch& S = ctx->inc;
  *done = false;
  const int64_t nold = G.nV;
  if (nV <= nold || nV >= ((int64_t)1 << 31) - 1 || G.nseg != 1) return HCI_OK;
  cudaStream_t st = ctx->st;
  unsigned long long* missing = reinterpret_cast<unsigned long long*>(bp<char>(ctx->s_counter) + 24);
  int64_t* dtot = reinterpret_cast<int64_t*>(bp<char>(ctx->s_counter) + 40);
  const ulonglong2* Vn = reinterpret_cast<const ulonglong2*>(keys);
  HCI_TRY(ensure_buf(ctx, S.pos_old, (size_t)nold * 8));
  HCI_TRY(ensure_buf(ctx, S.mark, (size_t)nV * 8));
  HCI_CUDA(ctx, cudaMemsetAsync(S.mark.p, 0, (size_t)nV * 8, st));
  HCI_CUDA(ctx, cudaMemsetAsync(missing, 0, 8, st));
  HCI_LAUNCH(k_find_old, grid_for(nold, 256), 256, 0, st)(bp<ulonglong2>(G.keys), nold, Vn, nV,
                                                          bp<int64_t>(S.pos_old), bp<int64_t>(S.mark), missing);
  unsigned long long miss = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&miss, missing, 8, cudaMemcpyDeviceToHost, st));
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  if (miss) return HCI_OK;        // not an extension: full rebuild
  prof_tic(ctx, HCI_PH_GRAPH);
  hci_status hs = HCI_OK;
  const int64_t nnew = nV - nold;
  // keys, maps and row arrays of the old space move to the scratch side
  std::swap(G.keys, S.keys_old);
  std::swap(G.s2i, S.s2i_old);
  std::swap(G.rowstart, S.rp_old);
  std::swap(G.rowlen, S.len_old);
  std::swap(G.rowcap, S.cap_old);
  HCI_TRY(ensure_buf(ctx, G.keys, (size_t)nV * 16));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.keys.p, keys, (size_t)nV * 16, cudaMemcpyDeviceToDevice, st));
  // new determinants in sorted order, their internal ids nold + q
  HCI_TRY(ensure_buf(ctx, S.flag, (size_t)(2 * nV + 1) * 8));
  int64_t* nflag = bp<int64_t>(S.flag);
  int64_t* npos = nflag + nV;
  HCI_LAUNCH(k_not, grid_for(nV, 256), 256, 0, st)(bp<int64_t>(S.mark), nV, nflag);
  HCI_TRY(scan_i64(ctx, nflag, npos, nV, dtot));
  HCI_TRY(ensure_buf(ctx, S.newrows, (size_t)nnew * 4));
  HCI_LAUNCH(k_compact_idx, grid_for(nV, 256), 256, 0, st)(nflag, npos, nV, bp<int32_t>(S.newrows));
  // maps and internal-order keys of V' (old ids and keys unchanged)
  HCI_TRY(ensure_buf(ctx, G.s2i, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, G.i2s, (size_t)nV * 4));
  HCI_TRY(grow_keep(ctx, G.keys_int, (size_t)nV * 16, (size_t)nold * 16));
  HCI_LAUNCH(k_build_perm, grid_for(nV, 256), 256, 0, st)(bp<int64_t>(S.pos_old), bp<int32_t>(S.s2i_old), nold,
                                                          bp<int32_t>(S.newrows), nnew, Vn, bp<int32_t>(G.s2i),
                                                          bp<int32_t>(G.i2s), bp<ulonglong2>(G.keys_int));
  GraphArgs A;
  HCI_TRY(build_space(ctx, nV, A));
  A.s2i = bp<int32_t>(G.s2i);
  A.rowlist = bp<int32_t>(S.newrows);
  A.nrows = nnew;
  prof_tic(ctx, HCI_PH_GRAPH_ROWS);
  // staging space from the mean length of a strided sample of the new rows
  // (the old rows' lengths say little when the space grows many-fold)
  int64_t nnzN = 0;
  {
    int64_t left = 0;
    HCI_TRY(stage_new_rows(ctx, A, nnew, nV, &nnzN, &left));
    HCI_TRY(ensure_buf(ctx, S.colN, (size_t)(nnzN + 1) * 4));
    HCI_TRY(ensure_buf(ctx, S.valN, (size_t)(nnzN + 1) * 8));
    HCI_TRY(stage_place(ctx, A, left, bp<int32_t>(S.colN)));
  }
  HCI_LAUNCH(k_row_values<true>, grid_for(nnew * 32, 256), 256, 0, st)(
      bp<int32_t>(S.newrows), nnew, bp<int64_t>(S.rpN), nullptr, bp<int32_t>(S.colN), bp<double>(S.valN),
      bp<ulonglong2>(G.keys), bp<ulonglong2>(G.keys_int), A.H);
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_GRAPH_ROWS);
  // transposed entries for the old rows, sorted by the row they go to
  prof_tic(ctx, HCI_PH_GRAPH_MERGE);
  HCI_TRY(ensure_buf(ctx, S.hist, (size_t)(nV + 1) * 8));
  HCI_CUDA(ctx, cudaMemsetAsync(S.hist.p, 0, (size_t)(nV + 1) * 8, st));
  const int gw = grid_for(nnew * 32, 256);
  HCI_LAUNCH(k_count_old_cols, gw, 256, 0, st)(bp<int64_t>(S.rpN), bp<int32_t>(S.colN), nnew, nold,
                                                bp<int64_t>(S.cnt), bp<int64_t>(S.hist));
  HCI_TRY(ensure_buf(ctx, S.tbase, (size_t)(nnew + 1) * 8));
  HCI_TRY(scan_i64(ctx, bp<int64_t>(S.cnt), bp<int64_t>(S.tbase), nnew, dtot));
  const int64_t nT = read_i64(ctx, dtot, &hs);
  HCI_TRY(hs);
  HCI_TRY(ensure_buf(ctx, S.T, (size_t)(nT + 1) * 16));
  HCI_TRY(ensure_buf(ctx, S.T2, (size_t)(nT + 1) * 16));
  HCI_LAUNCH(k_emit_T, gw, 256, 0, st)(bp<int64_t>(S.rpN), bp<int32_t>(S.colN), nnew, nold, bp<int64_t>(S.tbase),
                                        bp<ulonglong2>(S.T));
  int bits = 1;
  while (((int64_t)1 << bits) < nold) ++bits;
  HCI_TRY(sort_keys(ctx, bp<uint64_t>(S.T), bp<uint64_t>(S.T2), nT, bits, 0));
  HCI_TRY(ensure_buf(ctx, S.tstart, (size_t)(nV + 1) * 8));
  HCI_TRY(scan_i64(ctx, bp<int64_t>(S.hist), bp<int64_t>(S.tstart), nold, dtot));
  // plan the rows of V' (by internal id) in the pool: stay or take a new range
  HCI_TRY(ensure_buf(ctx, G.rowstart, (size_t)(nV + 1) * 8));
  HCI_TRY(ensure_buf(ctx, G.rowlen, (size_t)(nV + 1) * 8));
  HCI_TRY(ensure_buf(ctx, G.rowcap, (size_t)(nV + 1) * 8));
  HCI_TRY(ensure_buf(ctx, S.len, (size_t)(2 * nV + 2) * 8));
  int64_t* need = bp<int64_t>(S.len);
  int64_t* rel = need + nV + 1;
  int64_t total = 0;
  int repack = 0;
  for (int pass = 0; pass < 2; ++pass) {
    HCI_LAUNCH(k_plan_rows, grid_for(nV, 256), 256, 0, st)(
        bp<int64_t>(S.rp_old), bp<int64_t>(S.len_old), bp<int64_t>(S.cap_old), nold, bp<int64_t>(S.rpN), nnew,
        bp<int64_t>(S.hist), repack, bp<int64_t>(G.rowstart), bp<int64_t>(G.rowlen), bp<int64_t>(G.rowcap), need);
    HCI_TRY(scan_i64(ctx, need, rel, nV, dtot));
    total = read_i64(ctx, dtot, &hs);
    HCI_TRY(hs);
    if (repack || G.pool_used + total <= G.pool_cap) break;
    repack = 1;
  }
  int32_t* col_dst = bp<int32_t>(G.seg_col[0]);
  double* val_dst = bp<double>(G.seg_val[0]);
  int64_t base = G.pool_used;
  if (repack) {
    const int64_t cap = total + total / 4 + 1024;
    // the old pool stays alive while the new one is filled
    if (ctx->graph_budget > 0 && (cap + G.pool_cap) * 12 > ctx->graph_budget)
      return hci_fail(ctx, HCI_ERR_NOMEM, "graph: repacking into %lld bytes exceeds the budget of %lld",
                      (long long)(cap * 12), (long long)ctx->graph_budget);
    HCI_TRY(ensure_buf(ctx, S.col_old, (size_t)cap * 4));
    HCI_TRY(ensure_buf(ctx, S.val_old, (size_t)cap * 8));
    col_dst = bp<int32_t>(S.col_old);
    val_dst = bp<double>(S.val_old);
    base = 0;
  }
  HCI_LAUNCH(k_assign_starts, grid_for(nV, 256), 256, 0, st)(bp<int64_t>(G.rowstart), rel, nV, base);
  HCI_LAUNCH(k_move_old_rows, grid_for(nold * 32, 256), 256, 0, st)(
      bp<int64_t>(S.rp_old), bp<int64_t>(S.len_old), nold, bp<int32_t>(G.seg_col[0]), bp<double>(G.seg_val[0]),
      bp<int64_t>(G.rowstart), col_dst, val_dst, bp<ulonglong2>(S.T), bp<int64_t>(S.tstart), bp<int64_t>(S.hist),
      bp<double>(S.valN));
  HCI_LAUNCH(k_place_new_rows, gw, 256, 0, st)(nold, nnew, bp<int64_t>(S.rpN), bp<int32_t>(S.colN),
                                                bp<double>(S.valN), bp<int64_t>(G.rowstart), col_dst, val_dst);
  HCI_CUDA(ctx, cudaGetLastError());
  if (repack) {
    std::swap(G.seg_col[0], S.col_old);
    std::swap(G.seg_val[0], S.val_old);
    free_buf(st, S.col_old);
    free_buf(st, S.val_old);
    G.pool_cap = pool_entries(G);
    G.pool_used = total;
  } else {
    G.pool_used += total;
  }
  // logical prefix of the row lengths (internal order)
  HCI_TRY(ensure_buf(ctx, G.rowptr, (size_t)(nV + 1) * 8));
  HCI_TRY(scan_i64(ctx, bp<int64_t>(G.rowlen), bp<int64_t>(G.rowptr), nV, dtot));
  HCI_LAUNCH(k_store_at, 1, 1, 0, st)(bp<int64_t>(G.rowptr), nV, dtot);
  const int64_t nnz = read_i64(ctx, dtot, &hs);
  HCI_TRY(hs);
  prof_toc(ctx, HCI_PH_GRAPH_MERGE);
  if (nnz != G.nnz + nnzN + nT)
    return hci_fail(ctx, HCI_ERR_CUDA, "graph_extend: inconsistent sizes %lld != %lld + %lld + %lld", (long long)nnz,
                    (long long)G.nnz, (long long)nnzN, (long long)nT);
  // diagonal: old entries stay, the new ids are computed
  HCI_TRY(grow_keep(ctx, G.diag, (size_t)nV * 8, (size_t)nold * 8));
  HCI_TRY(compute_diag(ctx, nnew, bp<ulonglong2>(G.keys_int) + nold, bp<double>(G.diag) + nold));
  prof_toc(ctx, HCI_PH_GRAPH);
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  G.parent = G.epoch;
  G.epoch += 1;
  G.tail_entries = nnzN;
  G.nold = nold;
  G.nV = nV;
  G.nnz = nnz;
  G.nstored = nnz;
  ctx->st_counts[HCI_ST_GRAPH_BUILDS] += 1;
  *done = true;
  return HCI_OK;
}

// Direct form: the space's search structures and diagonal only (internal
// ids = sorted positions); every traversal searches the rows again.
static hci_status graph_build_direct(hci_ctx* ctx, const uint64_t* keys, int64_t nV) {
  Graph& G = ctx->graph;
  G.valid = false;
  free_segments(ctx);
  if (nV >= ((int64_t)1 << 31) - 1) return hci_fail(ctx, HCI_ERR_INVALID, "graph: nV exceeds int32 indices");
  prof_tic(ctx, HCI_PH_GRAPH);
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  HCI_TRY(ensure_buf(ctx, G.keys, (size_t)nV * 16));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.keys.p, keys, (size_t)nV * 16, cudaMemcpyDeviceToDevice, ctx->st));
  HCI_TRY(ensure_buf(ctx, G.keys_int, (size_t)nV * 16));
  HCI_CUDA(ctx, cudaMemcpyAsync(G.keys_int.p, keys, (size_t)nV * 16, cudaMemcpyDeviceToDevice, ctx->st));
  HCI_TRY(ensure_buf(ctx, G.s2i, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, G.i2s, (size_t)nV * 4));
  HCI_LAUNCH(k_iota, grid_for(nV, 256), 256, 0, ctx->st)(bp<int32_t>(G.s2i), bp<int32_t>(G.i2s), nV);
  GraphArgs A;
  HCI_TRY(build_space(ctx, nV, A));
  HCI_TRY(ensure_buf(ctx, G.diag, (size_t)nV * 8));
  HCI_TRY(compute_diag(ctx, nV, bp<ulonglong2>(G.keys_int), bp<double>(G.diag)));
  prof_toc(ctx, HCI_PH_GRAPH);
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  G.nV = nV;
  G.nnz = -1;   // counted by the first direct sigma
  G.direct = true;
  G.epoch += 1;
  G.parent = -1;
  ctx->st_counts[HCI_ST_GRAPH_BUILDS] += 1;
  G.valid = true;
  return HCI_OK;
}

// the stored rows and the incremental scratch, released before a direct build
static void release_stored(hci_ctx* ctx) {
  Graph& G = ctx->graph;
  IncScratch& S = ctx->inc;
  free_segments(ctx);
  DevBuf* bufs[] = {&G.rowptr, &G.rowstart, &G.rowlen, &G.rowcap, &S.scr, &S.stage, &S.grow, &S.col_old,
                    &S.val_old, &S.colN, &S.valN, &S.T, &S.T2};
  for (DevBuf* b : bufs) free_buf(ctx->st, *b);
  cudaStreamSynchronize(ctx->st);
}

// Stored form of the next build: both orientations unless the context was
// set to one orientation or fell back to it.
static bool want_half(const hci_ctx* ctx) {
  return ctx->sigma_mode == HCI_SIGMA_HALF || (ctx->sigma_mode == HCI_SIGMA_AUTO && ctx->half_fallback);
}

static hci_status graph_stored(hci_ctx* ctx, const uint64_t* keys, int64_t nV) {
  Graph& G = ctx->graph;
  const bool half = want_half(ctx);
  hci_status s = HCI_OK;
  bool done = false;
  if (G.valid && !G.direct && G.half == half && ctx->incremental) {
    G.valid = false;
    s = half ? graph_extend_half(ctx, keys, nV, &done) : graph_extend_full(ctx, keys, nV, &done);
  }
  if (s == HCI_OK && !done) {
    G.direct = false;
    s = half ? graph_build_half(ctx, keys, nV) : graph_build_full(ctx, keys, nV);
  }
  return s;
}

// HCI_SIGMA_AUTO: both orientations while they fit the budget (or device
// memory), then one orientation, then the direct form, each step for the
// rest of the context's life.
hci_status graph_ensure(hci_ctx* ctx, const uint64_t* keys, int64_t nV) {
  uint64_t hsh = 0;
  HCI_TRY(hash_keys(ctx, keys, nV, &hsh));
  if (ctx->graph.valid && ctx->graph.nV == nV && ctx->graph.hash == hsh) return HCI_OK;
  int ok = 0;
  HCI_TRY(check_sorted(ctx, keys, nV, &ok));
  if (!ok) return hci_fail(ctx, HCI_ERR_INVALID, "keys are not strictly ascending");
  const bool direct = ctx->sigma_mode == HCI_SIGMA_DIRECT || (ctx->sigma_mode == HCI_SIGMA_AUTO && ctx->direct_fallback);
  if (!direct) {
    hci_status s = graph_stored(ctx, keys, nV);
    if (s == HCI_ERR_NOMEM && ctx->sigma_mode == HCI_SIGMA_AUTO && !ctx->half_fallback) {
      // both orientations do not fit: store one orientation of each pair
      ctx->graph.valid = false;
      ctx->half_fallback = true;
      release_stored(ctx);
      s = graph_stored(ctx, keys, nV);
    }
    if (s == HCI_OK) {
      ctx->graph.hash = hsh;
      ctx->graph.valid = true;
      return HCI_OK;
    }
    if (s != HCI_ERR_NOMEM || ctx->sigma_mode != HCI_SIGMA_AUTO) return s;
    // the connections do not fit: search them again in every traversal
    ctx->graph.valid = false;
    ctx->direct_fallback = true;
    release_stored(ctx);
  }
  HCI_TRY(graph_build_direct(ctx, keys, nV));
  ctx->graph.hash = hsh;
  ctx->graph.valid = true;
  return HCI_OK;
}

// H c of a direct graph: every row's connections searched and evaluated
static hci_status sigma_direct(hci_ctx* ctx, const double* c, double* sigma, int nvec) {
  Graph& G = ctx->graph;
  GraphArgs A;
  space_args(ctx, G.nV, A);
  A.ddiag = bp<double>(G.diag);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(bp<char>(ctx->s_counter) + 56);
  for (int v = 0; v < nvec; ++v) {
    A.dc = c + (int64_t)v * G.nV;
    A.dsig = sigma + (int64_t)v * G.nV;
    A.dnnz = G.nnz < 0 ? cnt : nullptr;
    if (A.dnnz) HCI_CUDA(ctx, cudaMemsetAsync(cnt, 0, 8, ctx->st));
    HCI_CUDA(ctx, cudaMemsetAsync(A.queue, 0, 8, ctx->st));
    HCI_LAUNCH(k_rows<ROWS_SIGMA>, rows_grid(ctx), G_WARPS * 32, 0, ctx->st)(A);
    HCI_CUDA(ctx, cudaGetLastError());
    if (A.dnnz) {
      unsigned long long h = 0;
      HCI_CUDA(ctx, cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, ctx->st));
      HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
      G.nnz = (int64_t)h;
    }
  }
  return HCI_OK;
}

hci_status direct_rdm(hci_ctx* ctx, const double* c, const RdmAcc& R) {
  Graph& G = ctx->graph;
  GraphArgs A;
  space_args(ctx, G.nV, A);
  A.dc = c;
  A.R = R;
  HCI_CUDA(ctx, cudaMemsetAsync(A.queue, 0, 8, ctx->st));
  HCI_LAUNCH(k_rows<ROWS_RDM>, rows_grid(ctx), G_WARPS * 32, 0, ctx->st)(A);
  HCI_CUDA(ctx, cudaGetLastError());
  return HCI_OK;
}

hci_status sigma_apply(hci_ctx* ctx, const double* c, double* sigma, int nvec) {
  Graph& G = ctx->graph;
  if (G.direct) {
    prof_tic(ctx, HCI_PH_SIGMA);
    HCI_TRY(sigma_direct(ctx, c, sigma, nvec));
    ctx->st_counts[HCI_ST_SIGMA_CALLS] += nvec;
    ctx->st_counts[HCI_ST_SIGMA_ROWS] += G.nV * nvec;
    ctx->st_counts[HCI_ST_SIGMA_NNZ] += G.nnz * nvec;
    prof_toc(ctx, HCI_PH_SIGMA);
    return HCI_OK;
  }
  // one orientation: two passes when c and sigma together exceed half of L2
  // (HCI_SIGMA_HALF_PASSES set at context creation overrides the choice)
  const bool two_pass = G.half && nvec == 1 &&
                        (ctx->half_passes ? ctx->half_passes == 2 : (double)G.nV * 16.0 > 0.5 * (double)ctx->l2_bytes);
  if (G.half && !two_pass) HCI_CUDA(ctx, cudaMemsetAsync(sigma, 0, (size_t)G.nV * nvec * 8, ctx->st));
  prof_tic(ctx, HCI_PH_SIGMA);
  ctx->st_counts[HCI_ST_SIGMA_CALLS] += nvec;
  ctx->st_counts[HCI_ST_SIGMA_ROWS] += G.nV * nvec;
  ctx->st_counts[HCI_ST_SIGMA_NNZ] += G.nnz * nvec;
  if (G.half) {
    const SegTab T = G.tab();
    if (nvec == 1 && two_pass) {
      HCI_LAUNCH(k_sigma1_half<1>, ctx->nsm * SIGMA_HALF_BLOCKS_PER_SM, 256, 0, ctx->st)(
          bp<int64_t>(G.rowptr), bp<int64_t>(G.rowstart), T, bp<double>(G.diag), G.nV, c, sigma);
      HCI_LAUNCH(k_sigma1_half<2>, ctx->nsm * SIGMA_HALF_BLOCKS_PER_SM, 256, 0, ctx->st)(
          bp<int64_t>(G.rowptr), bp<int64_t>(G.rowstart), T, bp<double>(G.diag), G.nV, c, sigma);
    } else if (nvec == 1)
      HCI_LAUNCH(k_sigma1_half<0>, ctx->nsm * SIGMA_HALF_BLOCKS_PER_SM, 256, 0, ctx->st)(
          bp<int64_t>(G.rowptr), bp<int64_t>(G.rowstart), T, bp<double>(G.diag), G.nV, c, sigma);
    else
      HCI_LAUNCH(k_sigma_half, grid_for(G.nV * 32, 256, ctx->nsm * 16), 256, 0, ctx->st)(
          bp<int64_t>(G.rowptr), bp<int64_t>(G.rowstart), T, bp<double>(G.diag), G.nV, c, sigma, nvec);
  } else if (nvec == 1) {
    HCI_LAUNCH(k_sigma1, ctx->nsm * SIGMA_BLOCKS_PER_SM, 256, 0, ctx->st)(bp<int64_t>(G.rowptr), bp<int64_t>(G.rowstart),
                                                        bp<int32_t>(G.seg_col[0]), bp<double>(G.seg_val[0]),
                                                        bp<double>(G.diag), G.nV, c, sigma, 1);
  } else {
    HCI_LAUNCH(k_sigma, grid_for(G.nV * 32, 256, ctx->nsm * 16), 256, 0, ctx->st)(
        bp<int64_t>(G.rowptr), bp<int64_t>(G.rowstart), bp<int32_t>(G.seg_col[0]), bp<double>(G.seg_val[0]),
        bp<double>(G.diag), G.nV, c, sigma, nvec);
  }
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_SIGMA);
  return HCI_OK;
}

hci_status sigma_tail(hci_ctx* ctx, int64_t r0, const double* c, double* out) {
  Graph& G = ctx->graph;
  if (G.direct || r0 >= G.nV) return HCI_OK;
  HCI_LAUNCH(k_sigma_tail, grid_for((G.nV - r0) * 32, 256), 256, 0, ctx->st)(
      bp<int64_t>(G.rowptr), bp<int64_t>(G.rowstart), G.tab(), r0, G.nV, c, out);
  HCI_CUDA(ctx, cudaGetLastError());
  return HCI_OK;
}

hci_status to_internal(hci_ctx* ctx, const double* sorted, double* internal, int nvec) {
  const Graph& G = ctx->graph;
  HCI_LAUNCH(k_gather_vec, grid_for(G.nV * nvec, 256), 256, 0, ctx->st)(sorted, bp<int32_t>(ctx->graph.i2s), G.nV,
                                                                        nvec, internal);
  HCI_CUDA(ctx, cudaGetLastError());
  return HCI_OK;
}

hci_status to_sorted(hci_ctx* ctx, const double* internal, double* sorted, int nvec) {
  const Graph& G = ctx->graph;
  HCI_LAUNCH(k_gather_vec, grid_for(G.nV * nvec, 256), 256, 0, ctx->st)(internal, bp<int32_t>(ctx->graph.s2i), G.nV,
                                                                        nvec, sorted);
  HCI_CUDA(ctx, cudaGetLastError());
  return HCI_OK;
}

extern "C" hci_status hci_sigma(hci_ctx* ctx, const uint64_t* keys, int64_t nV, const double* c, double* sigma,
                                int nvec) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_sigma: null context");
  if (nV <= 0 || nvec <= 0) return hci_fail(ctx, HCI_ERR_INVALID, "hci_sigma: empty space or no vectors");
  if (!keys || !c || !sigma) return hci_fail(ctx, HCI_ERR_INVALID, "hci_sigma: null pointer");
  HCI_TRY(graph_ensure(ctx, keys, nV));
  HCI_TRY(ensure_buf(ctx, ctx->d_perm, (size_t)2 * nV * nvec * 8));
  double* ci = bp<double>(ctx->d_perm);
  double* si = ci + (int64_t)nV * nvec;
  HCI_TRY(to_internal(ctx, c, ci, nvec));
  HCI_TRY(sigma_apply(ctx, ci, si, nvec));
  return to_sorted(ctx, si, sigma, nvec);
}
