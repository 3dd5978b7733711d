// FP64 Davidson for the lowest eigenpair on a fixed determinant space:
// the minimum of the energy functional Eq. (variational) with the
// normalisation multiplier (Sec. II.A: after each enlargement of V the new
// ground state is found with Davidson's method).  Vector operations, the subspace eigenproblem
// (cyclic Jacobi on one warp) and the phase convention all run on the GPU;
// the host only reads the Ritz value and the residual norm per iteration.
#include <cmath>

#include "hci_internal.cuh"

namespace {

constexpr int MAXSUB = 24;          // subspace size before restart (<= 32)
constexpr int DAV_KEEP = 4;         // Ritz vectors kept for the next, grown space
constexpr int LDG = 32;             // leading dimension of the subspace matrix
constexpr int DBLOCK = 256;

struct DavDev {
  double G[LDG * LDG];
  double Qp[LDG * LDG];   // eigenvectors of the previous subspace matrix (kq x kq)
  double y[LDG];
  double dots[LDG];
  double ev[LDG];         // eigenvalues of the subspace matrix (columns of Qp)
  double theta;
  double nrm2;
  double ols[4];          // |r|^2, x . M^-1 r, x . M^-1 x (Olsen correction)
  int amax_idx;
  int kq;                 // size of Qp (0: none)
  unsigned int ticket;    // blocks of the running k_dots that have finished
  int stall;              // a correction fell inside the subspace (k_scale_unit)
};

// out[j] = V_j . w (j < k).  Each block writes partial[b][j], its share of
// the sums; the vectors come in groups of DOTS_GROUP (blockIdx.y = group),
// which keeps the accumulators few and the kernel at full occupancy for any
// k.  The last block to finish (a ticket counter) sums the partials in a
// fixed order (lanes over blocks, then a shuffle tree), so the
// result does not depend on the order in which blocks finish; with
// gcol >= 0 it also stores out[j] as G[j][gcol] = G[gcol][j], j <= gcol.
constexpr int DOTS_GROUP = 8;

__global__ void __launch_bounds__(DBLOCK) k_dots(const double* __restrict__ V, int64_t ld, int k,
                                                 const double* __restrict__ w, int64_t n, double* __restrict__ partial,
                                                 double* __restrict__ out, DavDev* __restrict__ gd, int gcol) {
  const int j0 = blockIdx.y * DOTS_GROUP;
  const int kg = k - j0 < DOTS_GROUP ? k - j0 : DOTS_GROUP;
  const double* Vg = V + (int64_t)j0 * ld;
  double acc[DOTS_GROUP];
#pragma unroll
  for (int j = 0; j < DOTS_GROUP; ++j) acc[j] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double wv = w[i];
#pragma unroll
    for (int j = 0; j < DOTS_GROUP; ++j)
      if (j < kg) acc[j] = fma(Vg[(int64_t)j * ld + i], wv, acc[j]);
  }
  __shared__ double red[DBLOCK / 32][DOTS_GROUP];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < DOTS_GROUP; ++j) {
    if (j < kg) {
      double a = acc[j];
      for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) red[wid][j] = a;
    }
  }
  __syncthreads();
  if (threadIdx.x < kg) {
    double s = 0.0;
    for (int w2 = 0; w2 < DBLOCK / 32; ++w2) s += red[w2][threadIdx.x];
    partial[(int64_t)blockIdx.x * LDG + j0 + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&gd->ticket, 1u) == gridDim.x * gridDim.y - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nblocks = (int)gridDim.x;
  for (int j = wid; j < k; j += DBLOCK / 32) {
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += __ldcg(partial + (int64_t)b * LDG + j);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      out[j] = s;
      if (gcol >= 0 && j <= gcol) {
        gd->G[j * LDG + gcol] = s;
        gd->G[gcol * LDG + j] = s;
      }
    }
  }
  if (threadIdx.x == 0) gd->ticket = 0u;
}

// Lowest eigenpair of the k x k subspace matrix by parallel-order Jacobi on
// one block of JW warps: in each round the indices are paired by a
// round-robin schedule and all disjoint pairs rotate at once (their
// rotations commute), so a sweep is k-1 rounds of parallel row and column
// updates, the pairs split over the warps.  An off-diagonal
// element too small to change either diagonal partner in floating point
// (even scaled by 100) is zeroed; the sweeps stop when a sweep rotates none.
//
// When the matrix is the previous one bordered by one row and column, the
// sweeps start from the previous eigenvectors Q0 = diag(Qp, 1): Q0^T G Q0 is
// diagonal but for its last row and column, and takes a few sweeps instead
// of a full diagonalisation.
constexpr int JW = 4;   // warps of k_jacobi: one per SM sub-partition (FP64 issue is the limit)

__global__ void __launch_bounds__(JW * 32) k_jacobi(DavDev* d, int k) {
  __shared__ double A[32][33];
  __shared__ double Q[32][33];
  __shared__ double T[32][33];
  __shared__ double rc[16], rs[16];
  __shared__ int rp[16], rq[16];
  __shared__ int s_rot, s_m;
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool warm = k > 1 && d->kq == k - 1;
  for (int j = w; j < 32; j += JW) {
    A[l][j] = (l < k && j < k) ? d->G[l * LDG + j] : 0.0;
    double q0 = (l == j) ? 1.0 : 0.0;
    if (warm && l < k - 1 && j < k - 1) q0 = d->Qp[l * LDG + j];
    Q[l][j] = q0;
  }
  __syncthreads();
  if (warm) {
    // T = G Q0 (lane = row, warps split the columns), then A = Q0^T T
    // (lane = column, warps split the rows)
    if (l < k)
      for (int j = w; j < k; j += JW) {
        double t = 0.0;
        for (int mm = 0; mm < k; ++mm) t = fma(A[l][mm], Q[mm][j], t);
        T[l][j] = t;
      }
    __syncthreads();
    if (l < k)
      for (int i = w; i < k; i += JW) {
        double t = 0.0;
        for (int mm = 0; mm < k; ++mm) t = fma(Q[mm][i], T[mm][l], t);
        A[i][l] = t;
      }
    __syncthreads();
  }
  const int m = (k + 1) & ~1;          // even number of players (index k is a dummy when k is odd)
  const int npairs = m / 2;
  for (int sweep = 0; sweep < 50 && k > 1; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < m - 1; ++r) {
      // thread t < npairs: pair t of round r
      if (threadIdx.x < npairs) {
        const int t = threadIdx.x;
        int a, b;
        if (t == 0) { a = r; b = m - 1; }
        else { a = (r + t) % (m - 1); b = (r - t + (m - 1)) % (m - 1); }
        int p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, sn = 0.0;
        int active = 0;
        if (q < k) {
          const double apq = A[p][q], app = A[p][p], aqq = A[q][q];
          const double g = 100.0 * fabs(apq);
          if (!((fabs(app) + g == fabs(app) && fabs(aqq) + g == fabs(aqq)) || fabs(apq) < 1e-300)) {
            // tan of the rotation angle, t = sgn(tau) / (|tau| + sqrt(1 +
            // tau^2)) with tau = (aqq - app) / (2 apq), written without the
            // division for tau (one square root, one division and one
            // reciprocal square root on this part's narrow FP64 pipe; the
            // entries are Rayleigh quotients of normalised vectors, far
            // from overflow)
            const double dd = aqq - app, e2 = 2.0 * apq;
            const double tt = copysign(1.0, dd) * e2 / (fabs(dd) + sqrt(dd * dd + e2 * e2));
            c = rsqrt(1.0 + tt * tt);
            sn = tt * c;
            active = 1;
          }
        }
        rp[t] = p; rq[t] = q; rc[t] = c; rs[t] = active ? sn : 0.0;
        if (!active && q < k) { A[p][q] = 0.0; A[q][p] = 0.0; }
        if (active) s_rot = 1;
      }
      __syncthreads();
      // columns: A <- A J, Q <- Q J (lane = row; warp w takes pairs w, w + JW, ...)
      if (l < k) {
        for (int t = w; t < npairs; t += JW) {
          const double s2 = rs[t];
          if (s2 == 0.0) continue;
          const int p = rp[t], q = rq[t];
          const double c2 = rc[t];
          const double alp = A[l][p], alq = A[l][q];
          A[l][p] = c2 * alp - s2 * alq;
          A[l][q] = s2 * alp + c2 * alq;
          const double vlp = Q[l][p], vlq = Q[l][q];
          Q[l][p] = c2 * vlp - s2 * vlq;
          Q[l][q] = s2 * vlp + c2 * vlq;
        }
      }
      __syncthreads();
      // rows: A <- J^T A (lane = column)
      if (l < k) {
        for (int t = w; t < npairs; t += JW) {
          const double s2 = rs[t];
          if (s2 == 0.0) continue;
          const int p = rp[t], q = rq[t];
          const double c2 = rc[t];
          const double apl = A[p][l], aql = A[q][l];
          A[p][l] = c2 * apl - s2 * aql;
          A[q][l] = s2 * apl + c2 * aql;
        }
      }
      __syncthreads();
      if (threadIdx.x < npairs && rs[threadIdx.x] != 0.0) {
        A[rp[threadIdx.x]][rq[threadIdx.x]] = 0.0;
        A[rq[threadIdx.x]][rp[threadIdx.x]] = 0.0;
      }
      __syncthreads();
    }
    const int rotated = s_rot;
    __syncthreads();
    if (!rotated) break;
  }
  if (threadIdx.x == 0) {
    int mm = 0;
    for (int j = 1; j < k; ++j)
      if (A[j][j] < A[mm][mm]) mm = j;
    s_m = mm;
    d->theta = A[mm][mm];
  }
  __syncthreads();
  const int mi = s_m;
  if (w == 0 && l < LDG) d->y[l] = (l < k) ? Q[l][mi] : 0.0;
  if (l < k)
    for (int j = w; j < k; j += JW) d->Qp[l * LDG + j] = Q[l][j];
  if (w == 0 && l < k) d->ev[l] = A[l][l];
  if (threadIdx.x == 0) d->kq = k;
}

// x = V y, wy = W y, r = wy - theta x, t = M^-1 r with M = theta - diag
// (guarded away from zero); partial[b][0..2] = block sums of r^2, x t and
// x M^-1 x for the Olsen correction.
__global__ void __launch_bounds__(DBLOCK) k_ritz(const double* __restrict__ V, const double* __restrict__ W, int64_t ld,
                                                 int k, DavDev* __restrict__ d, const double* __restrict__ diag,
                                                 int64_t n, double* __restrict__ x, double* __restrict__ wy,
                                                 double* __restrict__ t, double* __restrict__ partial) {
  __shared__ double ys[LDG];
  __shared__ double red[3][DBLOCK / 32];
  __shared__ bool s_last;
  if (threadIdx.x < LDG) ys[threadIdx.x] = d->y[threadIdx.x];
  __syncthreads();
  const double theta = d->theta;
  double acc = 0.0, axt = 0.0, axx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double xv = 0.0, wv = 0.0;
    for (int j = 0; j < k; ++j) {
      xv = fma(ys[j], V[(int64_t)j * ld + i], xv);
      wv = fma(ys[j], W[(int64_t)j * ld + i], wv);
    }
    double r = wv - theta * xv;
    double den = theta - diag[i];
    if (fabs(den) < 1e-8) den = den >= 0.0 ? 1e-8 : -1e-8;
    const double tv = r / den;
    x[i] = xv;
    wy[i] = wv;
    t[i] = tv;
    acc = fma(r, r, acc);
    axt = fma(xv, tv, axt);
    axx = fma(xv, xv / den, axx);
  }
  for (int o = 16; o; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    axt += __shfl_xor_sync(0xffffffffu, axt, o);
    axx += __shfl_xor_sync(0xffffffffu, axx, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = acc;
    red[1][threadIdx.x >> 5] = axt;
    red[2][threadIdx.x >> 5] = axx;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < DBLOCK / 32; ++w) s += red[threadIdx.x][w];
    partial[(int64_t)blockIdx.x * LDG + threadIdx.x] = s;
  }
  // the last block to finish sums the partials into ols[0..2] (as k_dots)
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&d->ticket, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < 3) {
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(partial + (int64_t)b * LDG + wid);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) d->ols[wid] = s;
  }
  if (threadIdx.x == 0) d->ticket = 0u;
}

// The kk <= DAV_KEEP lowest Ritz vectors of the current subspace (ascending Ritz value)
// and their H products: Qo[t] = sum_j Qp[j][o_t] V[j], Wo[t] likewise from W.
__global__ void __launch_bounds__(DBLOCK) k_keep(const double* __restrict__ V, const double* __restrict__ W,
                                                 int64_t ld, int k, const DavDev* __restrict__ d, int kk, int64_t n,
                                                 double* __restrict__ Qo, double* __restrict__ Wo) {
  __shared__ double ys[DAV_KEEP][LDG];
  __shared__ int order[DAV_KEEP];
  if (threadIdx.x == 0) {
    bool used[LDG];
    for (int j = 0; j < k; ++j) used[j] = false;
    for (int t = 0; t < kk; ++t) {
      int b = -1;
      for (int j = 0; j < k; ++j)
        if (!used[j] && (b < 0 || d->ev[j] < d->ev[b])) b = j;
      used[b] = true;
      order[t] = b;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk * k; e += blockDim.x) {
    const int t = e / k, j = e % k;
    ys[t][j] = d->Qp[j * LDG + order[t]];
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double qv[DAV_KEEP], wv[DAV_KEEP];
#pragma unroll
    for (int t = 0; t < DAV_KEEP; ++t) { qv[t] = 0.0; wv[t] = 0.0; }
    for (int j = 0; j < k; ++j) {
      const double vj = V[(int64_t)j * ld + i], wj = W[(int64_t)j * ld + i];
#pragma unroll
      for (int t = 0; t < DAV_KEEP; ++t)
        if (t < kk) {
          qv[t] = fma(ys[t][j], vj, qv[t]);
          wv[t] = fma(ys[t][j], wj, wv[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < DAV_KEEP; ++t)
      if (t < kk) {
        Qo[(int64_t)t * ld + i] = qv[t];
        Wo[(int64_t)t * ld + i] = wv[t];
      }
  }
}

// Spin-flip partners (S_z = 0 sector): partner[i] = internal id of the
// determinant with the alpha and beta strings of internal id i exchanged;
// *missing counts determinants whose partner is not in the space.
__global__ void k_flip_partner(const ulonglong2* __restrict__ keys_int, const ulonglong2* __restrict__ sorted,
                               const int32_t* __restrict__ s2i, int64_t n, int32_t* __restrict__ partner,
                               unsigned long long* __restrict__ missing) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ulonglong2 k = keys_int[i];
    const ulonglong2 f = make_ulonglong2(k.y, k.x);
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      const ulonglong2 m = sorted[mid];
      if (m.x < f.x || (m.x == f.x && m.y < f.y)) lo = mid + 1;
      else hi = mid;
    }
    if (lo < n && sorted[lo].x == f.x && sorted[lo].y == f.y) {
      partner[i] = s2i[lo];
    } else {
      partner[i] = -1;
      atomicAdd(missing, 1ull);
    }
  }
}

// Projection on spin parity p: v_i <- (v_i + p v_partner(i)) / 2, each pair
// once (from its lower id, both entries written); alpha = beta determinants
// keep v_i for p = +1 and vanish for p = -1.  The two entries of a pair end
// up with exactly equal magnitudes.
__global__ void k_parity_project(double* __restrict__ v, const int32_t* __restrict__ partner, int64_t n, double p) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = partner[i];
    if (j == i) {
      if (p < 0.0) v[i] = 0.0;
    } else if (j > i) {
      const double a = v[i], b = v[j];
      const double s = 0.5 * (a + p * b);
      v[i] = s;
      v[j] = p * s;
    }
  }
}

// Olsen correction: t = M^-1 (r - eps x) with eps = (x M^-1 r) / (x M^-1 x),
// which makes the correction orthogonal to x to first order.
__global__ void __launch_bounds__(DBLOCK) k_olsen(const DavDev* __restrict__ d, const double* __restrict__ diag,
                                                  int64_t n, const double* __restrict__ x, double* __restrict__ t) {
  const double den_x = d->ols[2];
  const double eps = den_x != 0.0 ? d->ols[1] / den_x : 0.0;
  const double theta = d->theta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double den = theta - diag[i];
    if (fabs(den) < 1e-8) den = den >= 0.0 ? 1e-8 : -1e-8;
    t[i] -= eps * x[i] / den;
  }
}

// v[i] += a * (a hash of i mapped to [-1, 1)): a start component in every
// symmetry sector (deflated roots need not share the lowest diagonal
// determinant's symmetry)
__global__ void k_add_hash(double* __restrict__ v, int64_t n, double a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t x = (uint64_t)i + 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    v[i] += a * ((double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  }
}

// t -= sum_j dots_j V_j
__global__ void k_orth(const double* __restrict__ V, int64_t ld, int k, const DavDev* __restrict__ d,
                       double* __restrict__ t, int64_t n) {
  __shared__ double cs[LDG];
  if (threadIdx.x < LDG) cs[threadIdx.x] = d->dots[threadIdx.x];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = t[i];
    for (int j = 0; j < k; ++j) v = fma(-cs[j], V[(int64_t)j * ld + i], v);
    t[i] = v;
  }
}

// x *= 1/sqrt(*s2) (and y likewise if given)
__global__ void k_scale_by(double* __restrict__ x, double* __restrict__ y, int64_t n, const double* __restrict__ s2) {
  double f = 1.0 / sqrt(*s2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] *= f;
    if (y) y[i] *= f;
  }
}

__global__ void k_scale_const(double* __restrict__ x, int64_t n, double f) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= f;
}

// y = x / sqrt(|x|^2) with |x|^2 = d->nrm2 read on the device (the
// normalised correction into its subspace slot); a correction of norm^2 at
// most 1e-26 lies in the subspace: y = 0 and d->stall = 1
__global__ void k_scale_unit(const double* __restrict__ x, int64_t n, DavDev* __restrict__ d, double* __restrict__ y) {
  const double nrm2 = d->nrm2;
  const bool ok = nrm2 > 1e-26;
  const double f = ok ? 1.0 / sqrt(nrm2) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = ok ? x[i] * f : 0.0;
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) d->stall = 1;
}

// argmax |x| (first index on ties): block partials then a final reduce
__global__ void k_amax_part(const double* __restrict__ x, int64_t n, double* __restrict__ pv, int64_t* __restrict__ pi) {
  double bv = -1.0;
  int64_t bi = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = fabs(x[i]);
    if (a > bv || (a == bv && i < bi)) { bv = a; bi = i; }
  }
  for (int o = 16; o; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  __shared__ double sv[32];
  __shared__ int64_t si[32];
  if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = bv; si[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] > bv || (sv[w] == bv && si[w] < bi)) { bv = sv[w]; bi = si[w]; }
    pv[blockIdx.x] = bv;
    pi[blockIdx.x] = bi;
  }
}

__global__ void k_phase_sign(const double* __restrict__ x, const double* __restrict__ pv,
                             const int64_t* __restrict__ pi, int nb, double* __restrict__ sgn) {
  double bv = -1.0;
  int64_t bi = 0;
  for (int b = 0; b < nb; ++b)
    if (pv[b] > bv || (pv[b] == bv && pi[b] < bi)) { bv = pv[b]; bi = pi[b]; }
  *sgn = x[bi] < 0.0 ? -1.0 : 1.0;
}

__global__ void k_apply_sign(double* __restrict__ x, int64_t n, const double* __restrict__ sgn) {
  const double s = *sgn;
  if (s > 0.0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = -x[i];
}

__global__ void k_unit_min_diag(double* __restrict__ x, const double* __restrict__ diag, int64_t n) {
  // single block: index of the smallest diagonal element (first on ties)
  double bv = 1e300;
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double a = diag[i];
    if (a < bv || (a == bv && i < bi)) { bv = a; bi = i; }
  }
  __shared__ double sv[1024];
  __shared__ int64_t si[1024];
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 1; t < (int)blockDim.x; ++t)
      if (sv[t] < bv || (sv[t] == bv && si[t] < bi)) { bv = sv[t]; bi = si[t]; }
    x[bi] = 1.0;
  }
}

struct Dav {
  hci_ctx* ctx;
  int64_t n, ld;
  double *V, *W, *x, *wy, *t, *part;
  DavDev* d;
  int nblk;

  // out[j] = Vb_j . w, j < k; with gcol >= 0 also column gcol of G
  hci_status dots(const double* Vb, int k, const double* w, double* out, int gcol = -1) {
    const dim3 grid((unsigned)nblk, (unsigned)((k + DOTS_GROUP - 1) / DOTS_GROUP));
    HCI_LAUNCH(k_dots, grid, DBLOCK, 0, ctx->st)(Vb, ld, k, w, n, part, out, d, gcol);
    HCI_CUDA(ctx, cudaGetLastError());
    return HCI_OK;
  }
  hci_status sigma(int slot) { return sigma_apply(ctx, V + (int64_t)slot * ld, W + (int64_t)slot * ld, 1); }
};

}  // namespace

// Spin-flip partners of the cached space (built once per graph epoch);
// HCI_ERR_INVALID when the space is not closed under the flip.
static hci_status parity_prepare(hci_ctx* ctx, int64_t nV) {
  const Graph& G = ctx->graph;
  if (ctx->partner_epoch == G.epoch && ctx->d_partner.bytes >= (size_t)nV * 4) return HCI_OK;
  HCI_TRY(ensure_buf(ctx, ctx->d_partner, (size_t)nV * 4));
  HCI_TRY(ensure_buf(ctx, ctx->s_counter, 64));
  unsigned long long* miss = reinterpret_cast<unsigned long long*>(bp<char>(ctx->s_counter) + 8);
  HCI_CUDA(ctx, cudaMemsetAsync(miss, 0, 8, ctx->st));
  HCI_LAUNCH(k_flip_partner, grid_for(nV, 256), 256, 0, ctx->st)(
      reinterpret_cast<const ulonglong2*>(G.keys_int.p), reinterpret_cast<const ulonglong2*>(G.keys.p),
      reinterpret_cast<const int32_t*>(G.s2i.p), nV, bp<int32_t>(ctx->d_partner), miss);
  HCI_CUDA(ctx, cudaGetLastError());
  unsigned long long h = 0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&h, miss, 8, cudaMemcpyDeviceToHost, ctx->st));
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  if (h) return hci_fail(ctx, HCI_ERR_INVALID, "spin parity: %llu determinants of V lack their spin-flip partner", h);
  ctx->partner_epoch = G.epoch;
  return HCI_OK;
}

static void parity_project(hci_ctx* ctx, double* v, int64_t nV, int nblk) {
  if (ctx->spin_parity == 0) return;
  HCI_LAUNCH(k_parity_project, nblk, DBLOCK, 0, ctx->st)(v, bp<int32_t>(ctx->d_partner), nV,
                                                        (double)ctx->spin_parity);
}

// The Davidson loop; with m > 0 locked vectors L (orthonormal, internal
// order, leading dimension (nV + 31) & ~31) the start vector and every
// correction are kept orthogonal to them, so the iteration converges to the
// lowest eigenpair of H in their complement (the next root when L holds the
// lower ones).
static hci_status davidson_core(hci_ctx* ctx, const uint64_t* keys, int64_t nV, double* c_inout, double* energy,
                                double tol, int maxit, int* iters, const double* L, int m) {
  if (iters) *iters = 0;
  HCI_TRY(graph_ensure(ctx, keys, nV));
  if (ctx->spin_parity != 0) HCI_TRY(parity_prepare(ctx, nV));
  prof_tic(ctx, HCI_PH_DAVIDSON);
  Dav D;
  D.ctx = ctx;
  D.n = nV;
  D.ld = (nV + 31) & ~(int64_t)31;
  D.nblk = grid_for(nV, DBLOCK, ctx->nsm * 8);
  HCI_TRY(ensure_buf(ctx, ctx->d_vb, (size_t)D.ld * (MAXSUB + 3) * 8));
  HCI_TRY(ensure_buf(ctx, ctx->d_wb, (size_t)D.ld * MAXSUB * 8));
  HCI_TRY(ensure_buf(ctx, ctx->d_part, (size_t)(D.nblk + 1) * LDG * 8));
  HCI_TRY(ensure_buf(ctx, ctx->d_small, sizeof(DavDev) + (size_t)(D.nblk + 1) * 16));
  D.V = bp<double>(ctx->d_vb);
  D.W = bp<double>(ctx->d_wb);
  D.x = D.V + (int64_t)MAXSUB * D.ld;
  D.wy = D.x + D.ld;
  D.t = D.wy + D.ld;
  D.part = bp<double>(ctx->d_part);
  D.d = bp<DavDev>(ctx->d_small);
  double* amax_v = reinterpret_cast<double*>(bp<char>(ctx->d_small) + sizeof(DavDev));
  int64_t* amax_i = reinterpret_cast<int64_t*>(amax_v + D.nblk);
  const double* diag = bp<double>(ctx->graph.diag);
  cudaStream_t st = ctx->st;
  HCI_CUDA(ctx, cudaMemsetAsync(D.d, 0, sizeof(DavDev), st));
  // A single-root run on the space the last one converged on, or on a space
  // grown from it, starts from that run's lowest Ritz vectors (zero on the
  // new determinants) with their H products: the old rows of those are
  // unchanged and the new rows cost one pass over the new rows' entries per
  // vector, so the warm start is taken when that is at most one product.
  const Graph& G = ctx->graph;
  DavKeep& K = ctx->dkeep;
  // A zero start vector asks for a cold start: the kept vectors are not used.
  double c0n2 = 0.0;
  {
    HCI_TRY(D.dots(c_inout, 1, c_inout, &D.d->nrm2));
    HCI_CUDA(ctx, cudaMemcpyAsync(&c0n2, &D.d->nrm2, 8, cudaMemcpyDeviceToHost, st));
    HCI_CUDA(ctx, cudaStreamSynchronize(st));
  }
  const bool same = K.valid && K.epoch == G.epoch && K.nV == nV;
  const bool grown = K.valid && !G.direct && G.parent == K.epoch && G.nold == K.nV &&
                     (double)G.tail_entries * K.k <= (double)(G.nstored > 0 ? G.nstored : 1);
  int kwarm = (m == 0 && c0n2 > 0.0 && (same || grown)) ? K.k : 0;
  if (kwarm > 0) {
    for (int j = 0; j < kwarm; ++j) {
      double* vj = D.V + (int64_t)j * D.ld;
      double* wj = D.W + (int64_t)j * D.ld;
      HCI_CUDA(ctx, cudaMemcpyAsync(vj, bp<double>(K.Q) + (int64_t)j * K.ld, (size_t)K.nV * 8,
                                    cudaMemcpyDeviceToDevice, st));
      HCI_CUDA(ctx, cudaMemcpyAsync(wj, bp<double>(K.W) + (int64_t)j * K.ld, (size_t)K.nV * 8,
                                    cudaMemcpyDeviceToDevice, st));
      if (nV > K.nV) {
        HCI_CUDA(ctx, cudaMemsetAsync(vj + K.nV, 0, (size_t)(nV - K.nV) * 8, st));
        HCI_TRY(sigma_tail(ctx, K.nV, vj, wj));
      }
    }
    for (int j = 0; j < kwarm; ++j) {
      HCI_TRY(D.dots(D.V, j + 1, D.W + (int64_t)j * D.ld, D.d->dots, j));
    }
  }
  // start vector, in the graph's internal order (after the kept vectors)
  double* V0 = D.V + (int64_t)kwarm * D.ld;
  HCI_TRY(to_internal(ctx, c_inout, V0, 1));
  HCI_TRY(D.dots(V0, 1, V0, &D.d->nrm2));
  double nrm2 = 0.0;
  HCI_CUDA(ctx, cudaMemcpyAsync(&nrm2, &D.d->nrm2, 8, cudaMemcpyDeviceToHost, st));
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  if (ctx->spin_parity != 0 && nrm2 > 0.0 && std::isfinite(nrm2)) {
    // the start vector's part of the requested spin parity
    parity_project(ctx, V0, nV, D.nblk);
    HCI_TRY(D.dots(V0, 1, V0, &D.d->nrm2));
    HCI_CUDA(ctx, cudaMemcpyAsync(&nrm2, &D.d->nrm2, 8, cudaMemcpyDeviceToHost, st));
    HCI_CUDA(ctx, cudaStreamSynchronize(st));
    if (!(nrm2 > 1e-20)) nrm2 = 0.0;
  }
  if (!(nrm2 > 0.0) || !std::isfinite(nrm2)) {
    HCI_CUDA(ctx, cudaMemsetAsync(V0, 0, (size_t)nV * 8, st));
    HCI_LAUNCH(k_unit_min_diag, 1, 1024, 0, st)(V0, diag, nV);
    if (m > 0 || ctx->spin_parity != 0)
      HCI_LAUNCH(k_add_hash, D.nblk, DBLOCK, 0, st)(V0, nV, 1e-2 / std::sqrt((double)nV));
    if (ctx->spin_parity != 0) {
      parity_project(ctx, V0, nV, D.nblk);
      HCI_TRY(D.dots(V0, 1, V0, &D.d->nrm2));
      HCI_CUDA(ctx, cudaMemcpyAsync(&nrm2, &D.d->nrm2, 8, cudaMemcpyDeviceToHost, st));
      HCI_CUDA(ctx, cudaStreamSynchronize(st));
      if (!(nrm2 > 1e-20)) return hci_fail(ctx, HCI_ERR_INVALID, "hci_davidson: no state of spin parity %+d in V",
                                           ctx->spin_parity);
      HCI_LAUNCH(k_scale_const, D.nblk, DBLOCK, 0, st)(V0, nV, 1.0 / std::sqrt(nrm2));
    }
  } else {
    HCI_LAUNCH(k_scale_const, D.nblk, DBLOCK, 0, st)(V0, nV, 1.0 / std::sqrt(nrm2));
  }
  bool add_start = true;
  if (kwarm > 0) {
    // the start vector joins the kept ones only with what they do not span
    for (int pass = 0; pass < 2; ++pass) {
      HCI_TRY(D.dots(D.V, kwarm, V0, D.d->dots));
      HCI_LAUNCH(k_orth, D.nblk, DBLOCK, 0, st)(D.V, D.ld, kwarm, D.d, V0, nV);
    }
    HCI_TRY(D.dots(V0, 1, V0, &D.d->nrm2));
    HCI_CUDA(ctx, cudaMemcpyAsync(&nrm2, &D.d->nrm2, 8, cudaMemcpyDeviceToHost, st));
    HCI_CUDA(ctx, cudaStreamSynchronize(st));
    add_start = nrm2 > 1e-16;
    if (add_start) HCI_LAUNCH(k_scale_const, D.nblk, DBLOCK, 0, st)(V0, nV, 1.0 / std::sqrt(nrm2));
  }
  if (m > 0) {
    // start orthogonal to the locked vectors (else the unit vector at the
    // lowest diagonal element, made orthogonal)
    for (int attempt = 0; attempt < 2; ++attempt) {
      for (int pass = 0; pass < 2; ++pass) {
        HCI_TRY(D.dots(L, m, D.V, D.d->dots));
        HCI_LAUNCH(k_orth, D.nblk, DBLOCK, 0, st)(L, D.ld, m, D.d, D.V, nV);
      }
      HCI_TRY(D.dots(D.V, 1, D.V, &D.d->nrm2));
      HCI_CUDA(ctx, cudaMemcpyAsync(&nrm2, &D.d->nrm2, 8, cudaMemcpyDeviceToHost, st));
      HCI_CUDA(ctx, cudaStreamSynchronize(st));
      if (nrm2 > 1e-20) break;
      if (attempt == 1) return hci_fail(ctx, HCI_ERR_INVALID, "hci_davidson_roots: no start vector outside the roots");
      HCI_CUDA(ctx, cudaMemsetAsync(D.V, 0, (size_t)nV * 8, st));
      HCI_LAUNCH(k_unit_min_diag, 1, 1024, 0, st)(D.V, diag, nV);
      HCI_LAUNCH(k_add_hash, D.nblk, DBLOCK, 0, st)(D.V, nV, 1e-2 / std::sqrt((double)nV));
      parity_project(ctx, D.V, nV, D.nblk);
    }
    HCI_LAUNCH(k_scale_const, D.nblk, DBLOCK, 0, st)(D.V, nV, 1.0 / std::sqrt(nrm2));
  }
  int k = kwarm;
  if (add_start) {
    HCI_TRY(D.sigma(k));
    HCI_TRY(D.dots(D.V, k + 1, D.W + (int64_t)k * D.ld, D.d->dots, k));
    ++k;
  }
  bool converged = false;
  double theta = 0.0, rn = 0.0;
  int it = 0;
  // one host synchronisation per iteration: the Ritz value, the residual
  // and whether the previous correction fell inside the subspace
  auto ritz = [&](double& th, double& r, int& stall) -> hci_status {
    HCI_LAUNCH(k_jacobi, 1, JW * 32, 0, st)(D.d, k);
    HCI_LAUNCH(k_ritz, D.nblk, DBLOCK, 0, st)(D.V, D.W, D.ld, k, D.d, diag, nV, D.x, D.wy, D.t, D.part);
    HCI_CUDA(ctx, cudaGetLastError());
    double hv[2];
    HCI_CUDA(ctx, cudaMemcpyAsync(&hv[0], &D.d->theta, 8, cudaMemcpyDeviceToHost, st));
    HCI_CUDA(ctx, cudaMemcpyAsync(&hv[1], &D.d->ols[0], 8, cudaMemcpyDeviceToHost, st));
    HCI_CUDA(ctx, cudaMemcpyAsync(&stall, &D.d->stall, 4, cudaMemcpyDeviceToHost, st));
    HCI_CUDA(ctx, cudaStreamSynchronize(st));
    th = hv[0];
    r = std::sqrt(hv[1]);
    return HCI_OK;
  };
  for (; it < maxit; ++it) {
    int stall = 0;
    HCI_TRY(ritz(theta, rn, stall));
    if (stall) {
      // the last correction lay in the subspace (it was added as zeros):
      // drop it, take the Ritz pair of the subspace before it and stop
      --k;
      HCI_TRY(ritz(theta, rn, stall));
      if (!std::isfinite(theta) || !std::isfinite(rn))
        return hci_fail(ctx, HCI_ERR_CUDA, "hci_davidson: non-finite Ritz value or residual");
      converged = rn <= tol;
      break;
    }
    if (!std::isfinite(theta) || !std::isfinite(rn))
      return hci_fail(ctx, HCI_ERR_CUDA, "hci_davidson: non-finite Ritz value or residual");
    if (rn <= tol) {
      converged = true;
      break;
    }
    if (k == MAXSUB) {
      // restart from the current Ritz vector
      HCI_CUDA(ctx, cudaMemcpyAsync(D.V, D.x, (size_t)nV * 8, cudaMemcpyDeviceToDevice, st));
      HCI_CUDA(ctx, cudaMemcpyAsync(D.W, D.wy, (size_t)nV * 8, cudaMemcpyDeviceToDevice, st));
      HCI_TRY(D.dots(D.V, 1, D.V, &D.d->nrm2));
      HCI_LAUNCH(k_scale_by, D.nblk, DBLOCK, 0, st)(D.V, D.W, nV, &D.d->nrm2);
      HCI_TRY(D.dots(D.V, 1, D.W, D.d->dots, 0));
      k = 1;
    }
    HCI_LAUNCH(k_olsen, D.nblk, DBLOCK, 0, st)(D.d, diag, nV, D.x, D.t);
    parity_project(ctx, D.t, nV, D.nblk);
    // orthogonalise the correction twice, normalise
    for (int pass = 0; pass < 2; ++pass) {
      HCI_TRY(D.dots(D.V, k, D.t, D.d->dots));
      HCI_LAUNCH(k_orth, D.nblk, DBLOCK, 0, st)(D.V, D.ld, k, D.d, D.t, nV);
      if (m > 0) {
        HCI_TRY(D.dots(L, m, D.t, D.d->dots));
        HCI_LAUNCH(k_orth, D.nblk, DBLOCK, 0, st)(L, D.ld, m, D.d, D.t, nV);
      }
    }
    HCI_TRY(D.dots(D.t, 1, D.t, &D.d->nrm2));
    double* slot = D.V + (int64_t)k * D.ld;
    HCI_LAUNCH(k_scale_unit, D.nblk, DBLOCK, 0, st)(D.t, nV, D.d, slot);
    HCI_TRY(D.sigma(k));
    HCI_TRY(D.dots(D.V, k + 1, D.W + (int64_t)k * D.ld, D.d->dots, k));
    ++k;
  }
  if (iters) *iters = it + (converged ? 1 : 0);
  // the lowest Ritz vectors for a later run on this space or a grown one
  K.valid = false;
  if (m == 0 && converged) {
    const int kk = k < DAV_KEEP ? k : DAV_KEEP;
    if (ensure_buf(ctx, K.Q, (size_t)D.ld * kk * 8) == HCI_OK && ensure_buf(ctx, K.W, (size_t)D.ld * kk * 8) == HCI_OK) {
      HCI_LAUNCH(k_keep, D.nblk, DBLOCK, 0, st)(D.V, D.W, D.ld, k, D.d, kk, nV, bp<double>(K.Q), bp<double>(K.W));
      K.valid = true;
      K.epoch = G.epoch;
      K.nV = nV;
      K.ld = D.ld;
      K.k = kk;
    }
  }
  // final vector: normalise, back to the caller's order, fix the phase
  // there (largest |c|, first sorted position on ties); with a spin parity
  // projected once more, so that the entries of a flip pair have equal
  // magnitudes exactly
  parity_project(ctx, D.x, nV, D.nblk);
  HCI_TRY(D.dots(D.x, 1, D.x, &D.d->nrm2));
  HCI_LAUNCH(k_scale_by, D.nblk, DBLOCK, 0, st)(D.x, nullptr, nV, &D.d->nrm2);
  HCI_TRY(to_sorted(ctx, D.x, c_inout, 1));
  HCI_LAUNCH(k_amax_part, D.nblk, DBLOCK, 0, st)(c_inout, nV, amax_v, amax_i);
  HCI_LAUNCH(k_phase_sign, 1, 1, 0, st)(c_inout, amax_v, amax_i, D.nblk, &D.d->dots[0]);
  HCI_LAUNCH(k_apply_sign, D.nblk, DBLOCK, 0, st)(c_inout, nV, &D.d->dots[0]);
  HCI_CUDA(ctx, cudaGetLastError());
  prof_toc(ctx, HCI_PH_DAVIDSON);
  HCI_CUDA(ctx, cudaStreamSynchronize(st));
  *energy = theta;
  if (!converged && rn > tol)
    return hci_fail(ctx, HCI_ERR_NOT_CONVERGED, "hci_davidson: residual %.3e > tol %.3e after %d iterations", rn, tol,
                    it);
  return HCI_OK;
}

extern "C" hci_status hci_set_spin_parity(hci_ctx* ctx, int parity) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_set_spin_parity: null context");
  if (parity < -1 || parity > 1) return hci_fail(ctx, HCI_ERR_INVALID, "hci_set_spin_parity: parity %d not in {-1, 0, 1}", parity);
  if (parity != 0 && ctx->na != ctx->nb)
    return hci_fail(ctx, HCI_ERR_INVALID, "hci_set_spin_parity: needs n_alpha = n_beta (S_z = 0), got %d and %d", ctx->na,
                    ctx->nb);
  if (parity != ctx->spin_parity) ctx->dkeep.valid = false;
  ctx->spin_parity = parity;
  return HCI_OK;
}

extern "C" hci_status hci_davidson(hci_ctx* ctx, const uint64_t* keys, int64_t nV, double* c_inout, double* energy,
                                   double tol, int maxit, int* iters) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_davidson: null context");
  if (nV <= 0 || !keys || !c_inout || !energy)
    return hci_fail(ctx, HCI_ERR_INVALID, "hci_davidson: empty space or null pointer");
  return davidson_core(ctx, keys, nV, c_inout, energy, tol, maxit, iters, nullptr, 0);
}

extern "C" hci_status hci_davidson_roots(hci_ctx* ctx, const uint64_t* keys, int64_t nV, int nroots, double* c_inout,
                                         double* energies, double tol, int maxit, int* iters) {
  if (!ctx) return hci_fail(nullptr, HCI_ERR_INVALID, "hci_davidson_roots: null context");
  if (nV <= 0 || !keys || !c_inout || !energies)
    return hci_fail(ctx, HCI_ERR_INVALID, "hci_davidson_roots: empty space or null pointer");
  if (nroots < 1 || nroots > nV || nroots > LDG)
    return hci_fail(ctx, HCI_ERR_INVALID, "hci_davidson_roots: nroots must lie in [1, min(nV, %d)]", LDG);
  if (iters) *iters = 0;
  HCI_TRY(graph_ensure(ctx, keys, nV));
  const int64_t ld = (nV + 31) & ~(int64_t)31;
  HCI_TRY(ensure_buf(ctx, ctx->d_lock, (size_t)ld * nroots * 8));
  double* L = bp<double>(ctx->d_lock);
  int total = 0;
  for (int r = 0; r < nroots; ++r) {
    int it = 0;
    hci_status s = davidson_core(ctx, keys, nV, c_inout + (int64_t)r * nV, &energies[r], tol, maxit, &it, L, r);
    total += it;
    if (iters) *iters = total;
    if (s != HCI_OK) return s;
    HCI_TRY(to_internal(ctx, c_inout + (int64_t)r * nV, L + (int64_t)r * ld, 1));
  }
  HCI_CUDA(ctx, cudaStreamSynchronize(ctx->st));
  return HCI_OK;
}
