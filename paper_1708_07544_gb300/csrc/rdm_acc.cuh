// Accumulation of one connected pair <D_i| op |D_j> into the spin-summed
// 1- and 2-RDMs (Sec. IV), shared by the stored-connection and the
// recomputing traversals.
#pragma once

#include "hci_internal.cuh"

__device__ __forceinline__ void add2(double* r2, int n, int p, int q, int r, int s, double v) {
  atomicAdd(&r2[(((int64_t)p * n + q) * n + r) * n + s], v);
}

// One orientation of every connected pair (column id above the row id): the
// other orientation contributes the transpose (p,q,r,s) -> (q,p,s,r), added
// in k_rdm_finish.  Doubles go to Hh (n^4).  A single a -> b of spin S in
// D_j with weight w adds w to S1[S][b][a]; its spectator terms
// sum w n_k(D_j) are split into the aufbau occupation (expanded in
// k_rdm_finish) plus the orbitals where D_j's strings differ from the
// aufbau ones, accumulated in Dt[b][a][k] (both spins) and Dx[b][a][k]
// (same spin, for the exchange terms).
struct RdmAcc {
  double* Hh;
  double* S1;
  double* Dt;
  double* Dx;
  uint64_t ref_a, ref_b;
};

// <ki| op |kj> of one connected pair (a single or double excitation apart)
// with weight cc, accumulated into R (doubles into Hh, singles into S1 / Dt /
// Dx as described above)
__device__ __forceinline__ void rdm_accumulate(const RdmAcc& R, int n, ulonglong2 ki, ulonglong2 kj, double cc) {
  const uint64_t xa = ki.x ^ kj.x, xb = ki.y ^ kj.y;
  const int da = __popcll(xa), db = __popcll(xb);
  if (da + db == 2) {
    // single a -> b in spin S
    const int S = da == 2 ? 0 : 1;
    const uint64_t sj = S == 0 ? kj.x : kj.y, oj = S == 0 ? kj.y : kj.x;
    const uint64_t x = S == 0 ? xa : xb;
    const int a = __ffsll((long long)(sj & x)) - 1;
    const int bb = __ffsll((long long)(x & ~sj)) - 1;
    const double w = cc * exc_phase(sj, a, bb);
    atomicAdd(&R.S1[((int64_t)S * n + bb) * n + a], w);
    const uint64_t rs = S == 0 ? R.ref_a : R.ref_b, ro = S == 0 ? R.ref_b : R.ref_a;
    double* dt = R.Dt + ((int64_t)bb * n + a) * n;
    double* dx = R.Dx + ((int64_t)bb * n + a) * n;
    for (uint64_t m = sj & ~rs; m; m &= m - 1) {
      const int kk = __ffsll((long long)m) - 1;
      atomicAdd(dt + kk, w);
      atomicAdd(dx + kk, w);
    }
    for (uint64_t m = rs & ~sj; m; m &= m - 1) {
      const int kk = __ffsll((long long)m) - 1;
      atomicAdd(dt + kk, -w);
      atomicAdd(dx + kk, -w);
    }
    for (uint64_t m = oj & ~ro; m; m &= m - 1) atomicAdd(dt + __ffsll((long long)m) - 1, w);
    for (uint64_t m = ro & ~oj; m; m &= m - 1) atomicAdd(dt + __ffsll((long long)m) - 1, -w);
  } else if (da == 4 || db == 4) {
    const uint64_t sj = da == 4 ? kj.x : kj.y;
    const uint64_t x = da == 4 ? xa : xb;
    uint64_t holes = sj & x, parts = x & ~sj;
    const int a = __ffsll((long long)holes) - 1; holes &= holes - 1;
    const int bh = __ffsll((long long)holes) - 1;
    const int cp = __ffsll((long long)parts) - 1; parts &= parts - 1;
    const int d = __ffsll((long long)parts) - 1;
    const double s1 = exc_phase(sj, a, cp);
    const uint64_t t = sj ^ (1ull << a) ^ (1ull << cp);
    const double w = cc * s1 * exc_phase(t, bh, d);
    add2(R.Hh, n, cp, a, d, bh, w);
    add2(R.Hh, n, d, bh, cp, a, w);
    add2(R.Hh, n, cp, bh, d, a, -w);
    add2(R.Hh, n, d, a, cp, bh, -w);
  } else {
    // alpha a -> c, beta b -> d
    const int a = __ffsll((long long)(kj.x & xa)) - 1, cp = __ffsll((long long)(ki.x & xa)) - 1;
    const int bh = __ffsll((long long)(kj.y & xb)) - 1, d = __ffsll((long long)(ki.y & xb)) - 1;
    const double w = cc * exc_phase(kj.x, a, cp) * exc_phase(kj.y, bh, d);
    add2(R.Hh, n, cp, a, d, bh, w);
    add2(R.Hh, n, d, bh, cp, a, w);
  }
}
