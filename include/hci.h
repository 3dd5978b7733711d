/*
 * hci.h -- C ABI of the GB300 (sm_103a) heat-bath CI active-space solver.
 *
 * Method: variational Heat-bath Configuration Interaction and the vHCISCF
 * orbital gradient of Smith, Mussard, Holmes & Sharma, "Cheap and near exact
 * CASSCF with large active spaces", arXiv:1708.07544 (Sec. II.A, III.B, IV).
 *
 * Problem statement (the active-space Hamiltonian handed to the solver,
 * Sec. III, Fig. 2):
 *   H = sum_pq h_pq sum_s a+_ps a_qs
 *     + 1/2 sum_pqrs (pq|rs) sum_st a+_ps a+_rt a_st a_qs + e_core
 * with real h (n x n, symmetric, row-major) and real (pq|rs) in chemists'
 * notation (n^4, row-major [p][q][r][s], exact 8-fold permutational
 * symmetry required: every permutation of one integral must hold the same
 * bits, because the heat-bath lists and the Slater-Condon rules read
 * different permutations).
 *
 * Determinants: keys[i] = { alpha bits, beta bits } as two uint64 words,
 * orbital p occupied <=> bit p set; norb <= 64.  A determinant is
 * prod_{alpha occ ascending} a+ prod_{beta occ ascending} a+ |0>.
 * Key arrays are [nV][2] uint64, 16-byte aligned, sorted strictly
 * ascending by (alpha, beta) (lexicographic, unsigned) unless stated.
 *
 * Memory and streams: every pointer argument marked "device" is device
 * memory owned by the caller; "host" pointers are host memory.  All work is
 * enqueued on the stream given to hci_create (a cudaStream_t passed as
 * void*; NULL = legacy default stream).  Calls that return a host scalar
 * synchronise that stream before returning.  The context owns only its
 * internal workspaces (integral tables, heat-bath lists, the connection
 * graph of the last space, scratch), allocated with cudaMallocAsync on the
 * context stream and released by hci_destroy to the device's default memory
 * pool, whose release threshold hci_create raises so that freed workspace
 * stays mapped for the next context (cudaMemPoolTrimTo returns it to the
 * system).  A context is not thread-safe.
 *
 * Errors: every call returns an hci_status.  On failure hci_last_error()
 * holds a one-line message.  HCI_ERR_CAPACITY reports, through the
 * call's size out-argument, the capacity that would have sufficed.
 */
#ifndef HCI_GB300_H
#define HCI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hci_ctx hci_ctx;
typedef int hci_status;

enum {
  HCI_OK = 0,
  HCI_ERR_INVALID = 1,        /* bad argument (norb > 64, counts, null, unsorted...) */
  HCI_ERR_CAPACITY = 2,       /* output buffer too small; required size returned */
  HCI_ERR_NOT_CONVERGED = 3,  /* Davidson reached maxit; outputs hold the last iterate */
  HCI_ERR_CUDA = 4,           /* a CUDA runtime call failed */
  HCI_ERR_NOMEM = 5           /* device allocation failed */
};

/* Create a solver for one active space.  h: device, n*n doubles; eri:
 * device, n^4 doubles (copied into the context, so the caller may free
 * them afterwards).  nalpha, nbeta in [0, norb], norb in [1, 64].
 * stream: cudaStream_t or NULL.  Derived tables for single-excitation
 * elements are built here.  (Sec. III, Fig. 2: each HCISCF iteration hands
 * the active-space one- and two-electron integrals to the HCI solver.) */
hci_status hci_create(hci_ctx** out, int norb, int nalpha, int nbeta, const double* h,
                      const double* eri, double e_core, void* stream);

/* Release the context and everything it owns (synchronises its stream). */
hci_status hci_destroy(hci_ctx* ctx);

/* Message of the last failure on this context ("" if none).  ctx may be
 * NULL, then the last failure of hci_create on this thread is returned. */
const char* hci_last_error(const hci_ctx* ctx);

/* Build the heat-bath excitation lists (Sec. II.A and Fig. 1b: double
 * excitation magnitudes depend only on the orbitals, so they are sorted and
 * stored before the run).  For every occupied opposite-spin pair (p_a, q_b)
 * the n^2 targets (r_a, s_b) with |(pr|qs)|, and for every same-spin pair
 * p<q the n(n-1)/2 targets r<s with |(pr|qs) - (ps|qr)|, each list sorted by
 * magnitude descending (ties by target ascending).  Idempotent. */
hci_status hci_build_lists(hci_ctx* ctx);

/* One selection step, Eq. (criteria) with the HCI importance function
 * f(D_a) = max_i |H_ai c_i| (Sec. II.A): every D_a not in V that is a single
 * or double excitation of some D_i in V with |H_ai| |c_i| > eps1 (strict;
 * eps1 <= 0 accepts every single and double).  Doubles come from the
 * heat-bath walk that stops at |v| <= eps1/|c_i|; singles are screened by
 * an upper bound and then evaluated exactly.
 *   keys: device [nV][2], sorted; c: device [nV] doubles;
 *   new_keys: device [cap][2] output, sorted, unique, disjoint from V;
 *   n_new: host out, number of new determinants (or the required cap on
 *   HCI_ERR_CAPACITY).  Builds the lists if needed.  Synchronises. */
hci_status hci_select(hci_ctx* ctx, double eps1, const uint64_t* keys, const double* c, int64_t nV,
                      uint64_t* new_keys, int64_t cap, int64_t* n_new);

/* V^{mu+1} = V^mu + C^mu (Sec. II.A): sorted union of two disjoint sorted
 * key sets.  out_keys: device [nV+n_new][2]; out_c: device [nV+n_new],
 * the old coefficients at their new positions and 0 for the new
 * determinants (Davidson warm start).  c and out_c may be NULL. */
hci_status hci_merge(hci_ctx* ctx, const uint64_t* keys, const double* c, int64_t nV,
                     const uint64_t* new_keys, int64_t n_new, uint64_t* out_keys, double* out_c);

/* sigma = H c on V for nvec vectors (Sec. II.A, the Davidson sigma; Sec. IV:
 * all single and double connections between pairs of determinants of V).
 * c, sigma: device, nvec column vectors of length nV stored one after the
 * other ([nvec][nV]).  The connection graph of V is built on first use and
 * cached until a call passes a different space (checked by content hash). */
hci_status hci_sigma(hci_ctx* ctx, const uint64_t* keys, int64_t nV, const double* c,
                     double* sigma, int nvec);

/* Lowest eigenpair on V, the minimum of the energy functional Eq.
 * (variational), by FP64 Davidson with a diagonal preconditioner.
 * c_inout: device [nV], the start vector on entry (zero => unit vector at
 * the lowest diagonal element), the normalised eigenvector on exit, with
 * its largest-magnitude component (lowest index on ties) positive.
 * energy: host out (includes e_core).  Converged when ||H c - E c||_2 <= tol.
 * iters: host out (may be NULL).  Synchronises.
 * The context keeps the four lowest Ritz vectors of a converged run (and
 * their H products); a later run with a non-zero start vector, on the same
 * space or on one grown from it by determinants appended since (the space
 * of the next selection step), starts from them together with the start
 * vector.  A zero start vector starts cold, from the unit vector alone. */
hci_status hci_davidson(hci_ctx* ctx, const uint64_t* keys, int64_t nV, double* c_inout,
                        double* energy, double tol, int maxit, int* iters);

/* Second-order Epstein-Nesbet correction with screening (Sec. II.B,
 * Eq. pt_hci):
 *   E2(eps2) = sum over D_a not in V of (sum'_i H_ai c_i)^2 / (e0 - H_aa),
 * the screened sum keeping the terms with |H_ai c_i| > eps2 (eps2 <= 0: every
 * single and double of V); D_a is in C(eps2) when one of its terms is kept.
 * keys: device [nV][2], strictly ascending; c: device [nV], the normalised
 * state on V; e0: its variational energy (including e_core).  The (target,
 * term) pairs are processed at once when they number at most max_pairs
 * (0: 2^28), else in hash classes of about max_pairs pairs; device memory
 * stays near 64 bytes x max_pairs.
 * e2: host out; n_ext: host out, |C(eps2)| (may be NULL).
 * Density matrices of the correction (Sec. V, Computational Details), in
 * the spin-summed order of hci_rdm12, with d_a = (sum'_i H_ai c_i) /
 * (e0 - H_aa) the first-order coefficients:
 *   rdm?_dd = sum over D_a in C(eps2) of d_a^2 <D_a| op |D_a>
 *   rdm?_dc = sum over the screened pairs of c_i d_a <D_i| op |D_a>
 * (the pairs are those of the screened sum: |H_ai c_i| > eps2).  rdm1_dd,
 * rdm1_dc: device [n][n]; rdm2_dd, rdm2_dc: device [n][n][n][n]; give all
 * four or none (NULL: not computed).  grad_c: device [nV] or NULL, the
 * derivative of E2 with respect to c at a fixed set of screened pairs,
 * 2 sum'_a d_a H_ai (the right-hand side of the z-vector equation, Sec.
 * III.A).  Synchronises.  Builds the heat-bath lists if needed. */
hci_status hci_pt2(hci_ctx* ctx, double eps2, const uint64_t* keys, const double* c, int64_t nV, double e0,
                   int64_t max_pairs, double* e2, int64_t* n_ext, double* rdm1_dd, double* rdm2_dd,
                   double* rdm1_dc, double* rdm2_dc, double* grad_c);

/* How sigma and the RDMs get the connections of V (Sec. IV builds them by
 * generating every single and double between pairs of V):
 *   HCI_SIGMA_STORED: stored once per space with both orientations of every
 *     connected pair (pooled CSR, int32 column + FP64 element, 12 bytes per
 *     ordered pair plus per-row slack), streamed by every H c as a pure
 *     gather; extended in place when V grows.
 *   HCI_SIGMA_HALF: stored with one orientation per pair (in the row of the
 *     later-inserted determinant; 12 bytes per pair, no slack: half the
 *     memory); every H c adds each entry to both of its rows, the second by
 *     an FP64 atomic add, so sums are taken in a run-dependent order; V's
 *     growth only appends rows.
 *   HCI_SIGMA_DIRECT: nothing stored; every H c and RDM pass searches the
 *     connections of each row again and evaluates their elements (a few
 *     hundred MB of search structures instead of ~12 bytes per connection,
 *     for spaces whose connections exceed device memory).
 *   HCI_SIGMA_AUTO (default): both orientations while the pool fits
 *     graph_budget bytes (0: device memory), else one orientation while that
 *     fits, else direct, each fallback for the rest of the context's life.
 * Results agree to rounding order.  Invalidates the cached graph.
 * HCI_ERR_INVALID for an unknown mode or a negative budget. */
enum { HCI_SIGMA_AUTO = 0, HCI_SIGMA_STORED = 1, HCI_SIGMA_DIRECT = 2, HCI_SIGMA_HALF = 3 };
hci_status hci_set_sigma_mode(hci_ctx* ctx, int mode, int64_t graph_budget);

/* Spin parity of the states sought in the S_z = 0 sector (n_alpha =
 * n_beta): the paper compares singlet and triplet states (Sec. VI), which
 * in that sector differ by their symmetry under the spin flip F (alpha and
 * beta strings exchanged; F |a, b> = (-1)^n_alpha |b, a>, and a state of
 * total spin S has F = (-1)^(n_alpha + S)).  parity = +1: even S
 * (singlets, quintets), -1: odd S (triplets), 0: no restriction (default).
 * With a parity set, hci_select adds the flip partner of every selected
 * determinant (so the space stays closed under F), and hci_davidson,
 * hci_davidson_roots, hci_solve and hci_solve_roots return states with
 * c(b, a) = parity c(a, b) (vectors projected on that sector; a zero start
 * vector starts from the lowest diagonal determinant plus a small fixed
 * hash, projected).  The first selection of hci_solve is made from the
 * aufbau determinant with c = [1] whatever its parity.  Davidson needs a
 * space closed under F (HCI_ERR_INVALID otherwise, or when it holds no
 * state of the parity).  HCI_ERR_INVALID for parity outside {-1, 0, 1} or
 * n_alpha != n_beta. */
hci_status hci_set_spin_parity(hci_ctx* ctx, int parity);

/* Semistochastic second-order correction (Sec. II.B, Eq. semistoc):
 *   E2(eps2) ~ E2^D(eps2_det) + mean_s [E2^S_s(eps2) - E2^S_s(eps2_det)],
 * E2^D the deterministic hci_pt2 value, and both stochastic terms of a
 * sample s evaluated on the same draws: n_draws determinants of V drawn
 * with replacement, D_i with probability p_i = W_i / sum W, W_i =
 * ceil(|c_i| 2^(B - E)) with 2^(E-1) <= max|c| < 2^E, B = 40 for nV <= 2^22
 * and 62 - ceil(log2 nV) above (p_i proportional to |c_i| to 2^-B).  Draw k of sample s takes the first word r of
 * Philox4x64-10 (Salmon et al., SC'11) at counter (k, s, 0, 0) and key
 * (seed, 0), u = floor(r sum W / 2^64), and the index i with
 * W_0 + .. + W_{i-1} <= u < W_0 + .. + W_i.  Each sample's estimate is the
 * unbiased multinomial estimator of the cited semistochastic HCI work: over
 * the targets D_a outside V of the drawn determinants' pairs kept by the
 * screen (|H_aj c_j| > eps), with x_j = H_aj c_j, f_j = w_j / p_j (w_j =
 * times drawn), S = sum f_j x_j, T = sum (f_j x_j)^2, U = sum f_j x_j^2:
 *   E2^S = sum_a (S^2 - T + (N_d - 1) U) / (N_d (N_d - 1) (e0 - H_aa)).
 * keys, c, e0, max_pairs: as hci_pt2 (keys strictly ascending, nV < 2^31).
 * eps2 <= eps2_det.  n_draws >= 2, n_samples >= 1, n_draws * n_samples <
 * 2^31.  result: host [3] = {estimate, its standard error over the samples
 * (0 for one sample), E2^D(eps2_det)}.  sample_e2: host [n_samples][2] =
 * {E2^S(eps2), E2^S(eps2_det)} per sample, or NULL.  draws: device int32
 * [n_samples][n_draws], the drawn indices into V, or NULL.  nV = 0 or
 * c = 0 give zeros.  Synchronises.  Builds the heat-bath lists if needed. */
hci_status hci_pt2_stochastic(hci_ctx* ctx, const uint64_t* keys, const double* c, int64_t nV, double e0,
                              double eps2, double eps2_det, int64_t n_draws, int n_samples, uint64_t seed,
                              int64_t max_pairs, double* result, double* sample_e2, int32_t* draws);

/* The z-vector equation of the HCISCF gradient (Sec. III.A, Eq. lagc): z
 * with (H - e0) z = P rhs on V and z orthogonal to c (P = 1 - c c^T), by
 * preconditioned conjugate gradients in the complement of c (H - e0 is
 * positive there when c is the lowest eigenvector; preconditioner
 * diag(H) - e0).  keys, c (normalised), rhs, z: device, sorted order.
 * Converged when ||P (rhs - (H - e0) z)||_2 <= tol; HCI_ERR_NOT_CONVERGED
 * after maxit iterations (z holds the last iterate).  iters: host out (may
 * be NULL).  Synchronises. */
hci_status hci_zvector(hci_ctx* ctx, const uint64_t* keys, int64_t nV, const double* c, double e0, const double* rhs,
                       double* z, double tol, int maxit, int* iters);

/* Relaxed density matrices of E_var + E2 (Sec. III.A, Eq. lambda) at a
 * fixed V and a fixed set of screened pairs: with d, g = dE2/dc and
 * Gamma^dd, Gamma^dc from hci_pt2 and z from hci_zvector(rhs = g),
 *   Gamma = (1 - |d|^2) Gamma(c) + Gamma^dd + Gamma^dc + (Gamma^dc)^T
 *           - 1/4 [Gamma(z + c) - Gamma(z - c)]
 * (and the same combination of the 1-RDMs), whose contraction with the
 * derivatives of h and (pq|rs) is d(E_var + E2); hci_rotate_backward maps
 * it to dE/dkappa.  c: the normalised lowest eigenvector on V, e0 its
 * energy.  e2: host out.  rdm1, rdm2: device, spin-summed order of
 * hci_rdm12.  Synchronises. */
hci_status hci_relaxed_rdm12(hci_ctx* ctx, double eps2, const uint64_t* keys, const double* c, int64_t nV, double e0,
                             int64_t max_pairs, double zv_tol, int zv_maxit, double* e2, double* rdm1,
                             double* rdm2);

/* <S^2> of a state from its spin-summed 2-RDM (rdm2 as hci_rdm12 writes it,
 * device [n][n][n][n]): -N (N - 4) / 4 - 1/2 sum_pq rdm2[p,q,q,p], which
 * follows from S^2 = S_z^2 + (S_+ S_- + S_- S_+) / 2 and the definition of
 * rdm2.  Tells the spin of the states of several roots (the paper's singlet
 * and triplet states, Sec. VI) apart within one S_z sector.  s2: host out.
 * Synchronises. */
hci_status hci_spin_square(hci_ctx* ctx, const double* rdm2, double* s2);

/* The nroots lowest eigenpairs on V (ascending), one after the other by
 * Davidson deflated against the converged lower ones (each start vector and
 * correction kept orthogonal to them).  c_inout: device [nroots][nV], start
 * vectors on entry (zero => unit vector at the lowest diagonal element, for
 * roots above the first plus 1e-2/sqrt(nV) times a fixed hash of each index
 * mapped to [-1, 1), so that no symmetry sector is missing from the start;
 * then made orthogonal), the normalised eigenvectors on exit (phase as
 * hci_davidson).
 * energies: host [nroots].  iters: host out, total iterations (may be NULL).
 * 1 <= nroots <= min(nV, 32).  Synchronises. */
hci_status hci_davidson_roots(hci_ctx* ctx, const uint64_t* keys, int64_t nV, int nroots, double* c_inout,
                              double* energies, double tol, int maxit, int* iters);

/* Variational HCI for the nroots lowest states (Sec. II.A): D_a enters when
 * max_r |H_ai c_i^(r)| > eps1, i.e. the selection with c_i replaced by
 * max_r |c_i^(r)|; V^0 = {aufbau}, then select, merge (every state padded
 * with zeros) and hci_davidson_roots (all states of V while it holds fewer
 * than nroots determinants) until the selection is empty; HCI_ERR_INVALID
 * when the final V is smaller than nroots.
 * keys_out: device [cap][2]; c_out: device with room for nroots * cap
 * doubles, written densely as [nroots][nV] (NULL allowed);
 * nV_out, energies [nroots], iters: host out.  HCI_ERR_CAPACITY when nV >
 * cap (nV_out holds the size). */
hci_status hci_solve_roots(hci_ctx* ctx, int nroots, double eps1, int max_iter, double dav_tol, int dav_maxit,
                           uint64_t* keys_out, double* c_out, int64_t cap, int64_t* nV_out, double* energies,
                           int* iters);

/* Spin-summed variational RDMs (Sec. IV, Gamma^{c,c}; accumulated over the
 * connections of V):
 *   rdm1[p*n+q]            = sum_s <a+_ps a_qs>
 *   rdm2[((p*n+q)*n+r)*n+s] = sum_st <a+_ps a+_rt a_st a_qs>
 * so that E = sum h rdm1 + 1/2 sum (pq|rs) rdm2 + e_core.  c must be
 * normalised for these to be expectation values.  rdm1, rdm2: device. */
hci_status hci_rdm12(hci_ctx* ctx, const uint64_t* keys, int64_t nV, const double* c, double* rdm1,
                     double* rdm2);

/* The whole variational stage (Sec. II.A, Fig. 1a): V^0 = {aufbau}, then
 * select / merge / Davidson until C^mu is empty or max_iter selections.
 * keys_out: device [cap][2]; c_out: device [cap]; nV: host out (required
 * cap on HCI_ERR_CAPACITY); energy: host out; iters: host out (selection
 * steps taken, may be NULL).  Synchronises. */
hci_status hci_solve(hci_ctx* ctx, double eps1, int max_iter, double dav_tol, int dav_maxit,
                     uint64_t* keys_out, double* c_out, int64_t cap, int64_t* nV, double* energy,
                     int* iters);

/* The variational stage resumed from a saved state (checkpoint and resume of
 * the selection loop of Sec. II.A: V^{mu+1} = V^mu + C^mu depends only on
 * V^mu and c^mu): keys0 (device [nV0][2], strictly ascending) and c0
 * (device [nV0], the state on that space, e.g. a step of an earlier solve
 * written to disk) stand for V^mu, c^mu; the next selection is made from
 * them as they are, then select / merge / Davidson as in hci_solve until the
 * selection is empty or max_iter more selections.  When the first selection
 * is already empty the state's energy comes from Davidson on (keys0, c0).
 * Outputs as hci_solve; iters counts the selections made here.  Synchronises. */
hci_status hci_solve_from(hci_ctx* ctx, const uint64_t* keys0, const double* c0, int64_t nV0, double eps1,
                          int max_iter, double dav_tol, int dav_maxit, uint64_t* keys_out, double* c_out, int64_t cap,
                          int64_t* nV, double* energy, int* iters);

/* Many independent active spaces of uneven size (a batch of orbital
 * iterations or of molecules; the paper solves one space per orbital
 * iteration, Sec. III): each
 * instance k gets its own context and stream, `nstreams` host threads take
 * instances from a shared queue, so uneven instances overlap on the GPU.
 * Arrays of length count: norb, nalpha, nbeta, h[k] / eri[k] (device
 * pointers as in hci_create), e_core (may be NULL = 0).  Outputs (host):
 * energies[k], nV[k] (size of the converged space), status[k] (may be
 * NULL).  rdm1 / rdm2 may be NULL, else arrays of device pointers receiving
 * each instance's RDMs (hci_rdm12 layout; a NULL entry skips that instance).
 * Returns the first failure (its instance named in hci_last_error(NULL));
 * the other instances still run.  Synchronises. */
hci_status hci_solve_batch(int count, const int* norb, const int* nalpha, const int* nbeta,
                           const double* const* h, const double* const* eri, const double* e_core, double eps1,
                           int max_iter, double dav_tol, int dav_maxit, int nstreams, double* energies,
                           int64_t* nV, double* const* rdm1, double* const* rdm2, int* status);

/* Active-active orbital rotation (Sec. III.A: the integrals depend on the
 * orbital parameters kappa; Sec. III.B): U = exp(kappa) for an n x n real
 * kappa (antisymmetric for an orthogonal U), h' = U^T h U,
 * (pq|rs)' = sum_abcd U_ap U_bq U_cr U_ds (ab|cd).
 * The outputs are made exactly symmetric, as hci_create requires: every
 * permutation of (pq|rs)' in its 8-fold orbit, and h'_qp, hold the bits of
 * the orbit's representative (p <= q, r <= s, pq <= rs) and of h'_pq, p < q.
 * All pointers device; U, h_out, eri_out are outputs (n*n, n*n, n^4).
 * stream: cudaStream_t or NULL. */
hci_status hci_rotate(int norb, const double* kappa, const double* h, const double* eri, double* U,
                      double* h_out, double* eri_out, void* stream);

/* One quarter transform of the rotation above (Sec. III.A), the n^5 part
 * of hci_rotate and hci_rotate_backward:
 *   out[J*n + p] = sum_a in[a*n^3 + J] * M[a*n + p],   J < n^3, p < n,
 * i.e. the summed index a leaves the front and p joins at the back (four
 * calls with M = U give (pq|rs)').  in and out are n^4 doubles, M is n*n,
 * all device pointers; in and out must not overlap.  Computed on the bf16
 * tensor cores as exact products of the balanced base-256 digits of each
 * row of in and each column of M (in fixed point against their largest
 * binary exponents), summed exactly and rounded once to FP64: the error is
 * at most about n 2^-55 of max_a |in[a][J]| * max_a |M[a][p]| (subnormal
 * entries count as zero).  Stream-ordered; with
 * check != 0 the call synchronises the stream and returns HCI_ERR_CUDA if
 * the launch gave up waiting for its products (never expected), which the
 * rotation entry points check after every call anyway. */
hci_status hci_qtrans(int norb, const double* in, const double* M, double* out, int check, void* stream);

/* Backward of E(h', eri') through the rotation, Eq. (vdedk2): given
 * dE/dh' = rdm1 and dE/d(pq|rs)' = rdm2/2 (Hellmann-Feynman at fixed V and
 * converged c), returns
 *   dh     = U rdm1 U^T                      (n*n)
 *   deri   = 1/2 sum rdm2_pqrs U_ap U_bq U_cr U_ds   (n^4)
 *   dkappa = dE/dkappa for every entry of the full kappa matrix (n*n),
 *            through the adjoint Frechet derivative of exp.
 * Any of dh, deri, dkappa may be NULL.  All pointers device.  Assumes the
 * 8-fold symmetry of eri and the pair symmetries of rdm2 of a real state. */
hci_status hci_rotate_backward(int norb, const double* kappa, const double* h, const double* eri,
                               const double* rdm1, const double* rdm2, double* dh, double* deri,
                               double* dkappa, void* stream);

/* hci_rotate without any device allocation (the paper has no counterpart:
 * this is a deployment variant).  For callers that cannot allocate device
 * memory when they need the rotation -- code inside another framework's
 * memory pool that forbids foreign allocations, or a host thread that must
 * not call cudaMalloc/cudaFree because those may synchronise the device.
 * Same arguments, outputs and results as hci_rotate; the caller still
 * provides every input and output buffer.  Scratch (one norb^4
 * intermediate and the exp(kappa) work matrices) lives in a static device
 * array of about 8 MiB that every GPU loading this library holds until the
 * process exits; norb above 32 is rejected with HCI_ERR_INVALID.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it for the CUDA context that is current;
 * a call made in another context (after a device reset, or from a context
 * the caller created) looks the address up again.  All calls share the
 * array: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * Synchronises the stream. */
hci_status hci_rotate_noalloc(int norb, const double* kappa, const double* h, const double* eri, double* U,
                              double* h_out, double* eri_out, void* stream);

/* Work counters of this context (instrumentation; the paper reports only
 * wall times per HCISCF iteration, Sec. V).  out[k] for k < nout:
 *   HCI_ST_GRAPH_NNZ        off-diagonal connections of the cached graph
 *                           (direct form: counted by its first product, 0
 *                           before)
 *   HCI_ST_LAST_CANDIDATES  candidates emitted by the last selection
 *   HCI_ST_SIGMA_CALLS      H c products so far (one per vector)
 *   HCI_ST_SIGMA_ROWS       rows processed by them
 *   HCI_ST_SIGMA_NNZ        off-diagonal connections processed by them
 *   HCI_ST_SELECT_CALLS     selection steps so far
 *   HCI_ST_SELECT_SOURCES   source determinants offered to them
 *   HCI_ST_CANDIDATES       candidates emitted by them in total
 *   HCI_ST_GRAPH_BUILDS     connection graphs built
 *   HCI_ST_WALK_ENTRIES     list entries examined by the heat-bath walks
 *   HCI_ST_SINGLES_EXACT    single excitations evaluated exactly
 *   HCI_ST_ROWS_REFILLED    new graph rows too long for the one-pass search,
 *                           filled by a second search
 *   HCI_ST_SIGMA_DIRECT     1 when the cached graph is direct (connections
 *                           searched again by every traversal), else 0
 *   HCI_ST_GRAPH_HALF       1 when the cached graph stores one orientation
 *                           of each pair, else 0 */
enum {
  HCI_ST_GRAPH_NNZ = 0, HCI_ST_LAST_CANDIDATES = 1, HCI_ST_SIGMA_CALLS = 2, HCI_ST_SIGMA_ROWS = 3,
  HCI_ST_SIGMA_NNZ = 4, HCI_ST_SELECT_CALLS = 5, HCI_ST_SELECT_SOURCES = 6, HCI_ST_CANDIDATES = 7,
  HCI_ST_GRAPH_BUILDS = 8, HCI_ST_WALK_ENTRIES = 9, HCI_ST_SINGLES_EXACT = 10, HCI_ST_ROWS_REFILLED = 11,
  HCI_ST_SIGMA_DIRECT = 12, HCI_ST_GRAPH_HALF = 13, HCI_ST_COUNT = 14
};
hci_status hci_stats(const hci_ctx* ctx, int64_t* out, int nout);

/* Phases timed by hci_profile / hci_timers. */
enum {
  HCI_PH_LISTS = 0,     /* heat-bath list build */
  HCI_PH_WALK = 1,      /* heat-bath walk over the double-excitation lists */
  HCI_PH_DEDUP = 2,     /* radix sort, set difference against V, compaction */
  HCI_PH_MERGE = 3,     /* sorted union V + C */
  HCI_PH_GRAPH = 4,     /* connection graph + diagonal of a new space */
  HCI_PH_SIGMA = 5,     /* the sigma kernel alone (one entry per H c product) */
  HCI_PH_DAVIDSON = 6,  /* hci_davidson excluding the graph build */
  HCI_PH_RDM = 7,       /* hci_rdm12 excluding the graph build */
  HCI_PH_SINGLES = 8,   /* single excitations of the selection */
  HCI_PH_GRAPH_SPACE = 9,  /* string groups, beta-major order, neighbour lists */
  HCI_PH_GRAPH_ROWS = 10,  /* row search and element evaluation */
  HCI_PH_GRAPH_MERGE = 11, /* incremental update: transposes and CSR merge */
  HCI_PH_RDM_DIAG = 12,    /* diagonal part of the RDMs */
  HCI_PH_HDIAG = 13,       /* diagonal Hamiltonian elements */
  HCI_PH_COUNT = 14
};

/* Enable (1) or disable (0) per-phase CUDA-event timing on the context
 * stream.  Instrumentation only: it adds event records, no host syncs. */
hci_status hci_profile(hci_ctx* ctx, int enable);

/* Read and reset the per-phase totals: ms[k] = summed device time of phase k
 * in milliseconds, counts[k] = number of timed intervals, for k < nphase
 * (<= HCI_PH_COUNT).  Synchronises the context stream. */
hci_status hci_timers(hci_ctx* ctx, double* ms, int64_t* counts, int nphase);

/* Number of kernels this library has launched in the process so far. */
int64_t hci_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* HCI_GB300_H */
