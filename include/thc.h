/*
 * thc.h -- C ABI of the GB300 (sm_103a) THC-MPO Krylov library.
 *
 * The library applies a tensor-hypercontraction (THC) factorised molecular
 * Hamiltonian to a matrix-product state (MPS) and recompresses the result,
 * the hot path of the THC-MPO Krylov method of arXiv 2409.12708.  Every
 * numerical step runs in this library's own CUDA kernels on one GPU.
 *
 * Conventions shared by all calls
 * -------------------------------
 *  - Pointers called "device" point to GPU memory of the current device;
 *    "host" pointers point to CPU memory.  Inputs are never modified.
 *  - All work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *    stream).  Calls that return scalars to the host (mps_inner, the Krylov
 *    drivers) synchronise `stream` before returning; the others return as soon
 *    as the work is enqueued, and their outputs are valid once `stream` reaches
 *    that point.
 *  - Errors: a call returns a thc_status.  THC_EINVAL means a shape, size or
 *    argument was rejected before any work was enqueued and no output was
 *    written.  Other non-OK statuses may leave outputs partially written.
 *    thc_last_error() returns a message for the last non-OK status of the
 *    calling thread.
 *  - Memory: outputs (thc_mps with owner != NULL) and internal workspace are
 *    obtained from the caller's thc_allocator (stream-ordered alloc/free
 *    callbacks); a NULL allocator means cudaMallocAsync/cudaFreeAsync on
 *    `stream`.  Workspace is released before the call returns (stream-ordered).
 *
 * MPS layout (Sec. 2.1, the MPS equation): L order-3 site tensors, site i has
 * shape [bond[i], d, bond[i+1]] stored row-major (right bond fastest), with
 * bond[0] = bond[L] = 1 and d = 4.  The local basis index is 2*n_up + n_dn
 * (App. C: b_up = c (x) I2, b_dn = Z (x) c, spin-up major).
 */
#ifndef THC_H
#define THC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define THC_MAX_SITES 64

typedef enum {
    THC_OK = 0,
    THC_EINVAL = 1,        /* bad argument / shape / dtype; nothing written          */
    THC_ENOMEM = 2,        /* allocator returned NULL                                 */
    THC_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed             */
    THC_ENONFINITE = 4,    /* a NaN/Inf was detected in an input or a result          */
    THC_ETIMEOUT = 5,      /* the small float64 eigensolver ran out of sweeps (a Jacobi
                              SVD that ends its sweep budget is counted in the
                              profile, not raised: untruncated, the projector
                              correction keeps the state exact; truncating, the
                              kept rows are orthogonal only to the last sweep's
                              largest rotation, so the result can be off)           */
    THC_EBREAKDOWN = 6,    /* Krylov breakdown: the Krylov space is exhausted         */
    THC_EUNSUPPORTED = 7   /* valid request this build does not implement             */
} thc_status;

/* Storage dtype of MPS site tensors. */
typedef enum { THC_F64 = 0, THC_F32 = 1, THC_C64 = 2, THC_C128 = 3 } thc_dtype;

/* Compute path.  FP64: every step in float64 ("plain FP64 path"); site tensors
 * F64, or C128 for complex MPS.  FP32: site tensors (F32 or C64),
 * contractions, QR and Jacobi SVD in float32; singular values are accumulated
 * and the truncation decided in float64; inner products and the Krylov
 * projected problems are float64.  Complex MPS (the states of a time
 * evolution, Sec. 2.2) take the same steps with complex Householder
 * reflectors, complex one-sided Jacobi rotations and conjugation on the bra;
 * they are supported up to D_max = 256 (THC_EUNSUPPORTED above).
 * TF32: FP32 storage (F32 or C64) and steps, except that the contractions of
 * the compression (the expand-and-absorb, centre, U and projector products)
 * of real MPS run on the tensor cores as error-compensated TF32 (each float32
 * operand split into two TF32 numbers, three products accumulated in float32,
 * Ootomo & Yokota 2022), which keeps float32 accuracy. */
typedef enum { THC_PATH_FP64 = 0, THC_PATH_FP32 = 1, THC_PATH_TF32 = 2 } thc_path;

/* Stream-ordered allocator supplied by the caller (e.g. PyTorch's caching
 * allocator).  alloc returns NULL on failure. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void  (*free)(void* ptr, void* stream, void* ctx);
    void* ctx;
} thc_allocator;

/* MPS descriptor.  For inputs the caller fills L, d, dtype, bond[0..L] and
 * site[0..L-1] (device pointers) and sets owner = NULL; the library reads the
 * site tensors only.  For outputs the library fills every field; all sites live
 * in one device block `owner` obtained from the allocator, released by
 * thc_mps_free. */
typedef struct {
    int L;
    int d;
    thc_dtype dtype;
    int bond[THC_MAX_SITES + 1];
    void* site[THC_MAX_SITES];
    void* owner;
} thc_mps;

/* THC-factorised Hamiltonian, Eq. 1 with Eq. thc: device float64 arrays,
 * row-major: t[L*L] (symmetric one-body integrals t_pq), chi[L*N]
 * (chi[p*N + mu] = chi^mu_p), zeta[N*N] (symmetric zeta^{mu nu}). */
typedef struct {
    int L;
    int N;
    const double* t;
    const double* chi;
    const double* zeta;
} thc_hamiltonian;

/* Options.  D_max: MPS bond cap after every compression (the paper's M).
 * tol: relative discarded-weight tolerance of the truncation (0 = cap only).
 * term_begin/term_end: half-open range of term indices to apply (-1 = all;
 * an empty range is THC_EINVAL);
 * Coulomb terms G_{mu s, nu s'} have index ((s'*N + nu)*2 + s)*N + mu and
 * kinetic terms T_{i s} index 4N^2 + s*L + i.  batch: terms in flight
 * (0 = choose from free memory).  chunk: at most this many term states are
 * held before their partial sum is formed (rounded down to a power of two, so
 * every chunk is a whole subtree of the pairwise reduction and the result does
 * not depend on it; 0 = as many as a quarter of free memory holds).
 * merge_spin (0 = off, 1 = on; every call that applies H, including the Krylov
 * calls; thc_expect_grad ignores it): fold the opposite-spin Coulomb terms
 * pairwise.  For s != s' the one-body operators G_{mu s} and G_{nu s'} act on
 * different spin modes and commute, so with zeta symmetric (Eq. thc) the terms
 * (mu down, nu up) sum to the same operator as (mu up, nu down); the merged
 * list keeps zeta^{mu nu} G_{mu up} G_{nu down} with twice the coefficient and
 * drops the other, 3N^2 Coulomb terms instead of 4N^2 (same-spin products do
 * not commute and stay).  Term indices then run block by block: t < N^2 is
 * block (nu = t / N, s' = up) with mu = t % N, s = up; for t' = t - N^2 < 2N^2,
 * block (nu = t' / 2N, s' = down), s = (t' / N) % 2, mu = t' % N; kinetic
 * terms follow at 3N^2 + s*L + i.  Exact when zeta = zeta^T (the caller's
 * responsibility); the truncated result differs from the unmerged one by
 * truncation error, as any change of the term list does. */
typedef struct {
    int D_max;
    double tol;
    thc_path path;
    long term_begin;
    long term_end;
    int batch;
    int chunk;
    int merge_spin;
} thc_opts;

/* H|psi> as a compressed MPS: Alg. 1 of the paper (the reuse of
 * G_{nu s'}|psi> across all (mu, s)), plus the kinetic terms of App. D; each of
 * the bond-2 ladder MPOs of the elementary-MPO equations is applied and
 * followed by the QR-then-SVD compression of Fig. 3, and the compressed terms
 * are summed by the pairwise reduction of Sec. 4.5.  psi must have dtype
 * F64 or C128 (path FP64), F32 or C64 (paths FP32 and TF32; complex MPS run
 * the TF32 path's contractions on the SIMT pipe).  `out` receives a
 * library-owned MPS of the same dtype whose bonds are at most D_max. */
thc_status thc_apply_H(const thc_hamiltonian* H, const thc_mps* psi, const thc_opts* opts,
                       thc_mps* out, const thc_allocator* alloc, void* stream);

/* Several independent H|psi> at once (e.g. instances of uneven L): out[i] =
 * thc_apply_H(H[i], psi[i]) for i < n, with one opts for all.  Every instance
 * runs on its own stream, forked from `stream` and joined back into it before
 * the call returns (so `stream` orders after all of them), driven by its own
 * host thread; their kernels run concurrently on the device.  With
 * opts->batch = 0 the terms in flight are split between the instances
 * (max(32, 4 * SMs / n) each).  H[i], psi[i]: as for thc_apply_H; all psi
 * share one dtype.  out: caller array of n descriptors, each filled with a
 * library-owned MPS.  On failure every output already made is released and the
 * first failing instance's status is returned (its message names it). */
thc_status thc_apply_H_batched(int n, const thc_hamiltonian* const* H, const thc_mps* const* psi,
                               const thc_opts* opts, thc_mps* out, const thc_allocator* alloc, void* stream);

/* One elementary MPO (a ladder operator sum_s coef_s a_{s,sigma}, or its
 * creation counterpart when dagger != 0) applied to psi and compressed
 * (Sec. 3.1, Fig. 3).  coef: device float64 [L]; sigma: 0 = up, 1 = down. */
thc_status thc_layer_apply(const thc_mps* psi, const double* coef, int sigma, int dagger,
                           const thc_opts* opts, thc_mps* out,
                           const thc_allocator* alloc, void* stream);

/* Compression of Fig. 3 alone: QR sweep to right-canonical form, then the
 * left-to-right SVD truncation sweep (no renormalisation). */
thc_status thc_compress(const thc_mps* psi, const thc_opts* opts, thc_mps* out,
                        const thc_allocator* alloc, void* stream);

/* <phi|psi> = sum conj(phi) psi by transfer matrices, accumulated in float64
 * (complex float64 for complex MPS).  phi and psi share L and dtype.
 * out_re / out_im: host pointers (out_im may be NULL; 0 for real states). */
thc_status mps_inner(const thc_mps* phi, const thc_mps* psi, double* out_re, double* out_im,
                     void* stream);

/* compress(sum_i coeff_i |x_i>): direct sums and compressions of the pairwise
 * reduction (Sec. 3.2, Sec. 4.5).  coeff_re/coeff_im: host float64 [n]
 * (coeff_im may be NULL; non-zero imaginary parts need complex MPS, else
 * THC_EINVAL).  All xs share L and dtype; their bonds are at most
 * min(D_max, 4^b, 4^(L-b)). */
thc_status mps_add_compress(int n, const double* coeff_re, const double* coeff_im,
                            const thc_mps* const* xs, const thc_opts* opts, thc_mps* out,
                            const thc_allocator* alloc, void* stream);

/* Lanczos ground state (Sec. 2.2): K Krylov vectors by Gram-Schmidt, the full
 * projected matrix Htil_jk = <v_j|H v_k> and overlap S_jk, the correction of
 * Eq. reortho / Eq. eff_H by canonical orthogonalisation, float64 eigensolver.
 * energy: host double; ritz: host double[K] (ascending Ritz values, unused
 * entries NaN; may be NULL); ground: optional output MPS of the Ritz vector
 * (NULL to skip).  Returns THC_EBREAKDOWN only if not even one vector exists. */
thc_status krylov_lanczos_ground(const thc_hamiltonian* H, const thc_mps* psi0, int K,
                                 const thc_opts* opts, double* energy, double* ritz,
                                 thc_mps* ground, const thc_allocator* alloc, void* stream);

/* Restarted Lanczos and excited states (Sec. 2.2: restarting improves the
 * convergence under truncation; an excited state follows from a start vector
 * orthogonal to the lower eigenstates).  `cycles` runs of the Lanczos of
 * krylov_lanczos_ground with K vectors each, every run started from the
 * previous run's lowest Ritz vector (its pairwise-reduced combination of the
 * v_i, normalised).  lower[0..n_lower-1]: optional orthonormal MPS (e.g. lower
 * eigenstates; same L and dtype as psi0, bonds at most min(D_max, 4^b,
 * 4^(L-b))): the start vector and every Krylov vector are orthogonalised
 * against them within the same Gram-Schmidt sum, so the lowest Ritz value
 * approximates the next level above them.  energies: host double[cycles],
 * the lowest Ritz value of each run; state: optional output MPS (psi0's
 * dtype), the last Ritz vector (NULL to skip).  Dense tensors conserve
 * (N_up, N_dn) only to rounding: over many Krylov vectors rounding noise in
 * other particle-number sectors can grow toward their lower levels.
 * Errors as krylov_lanczos_ground; THC_EINVAL for cycles < 1 or bad lower
 * states. */
thc_status krylov_lanczos_restarted(const thc_hamiltonian* H, const thc_mps* psi0, int K, int cycles,
                                    int n_lower, const thc_mps* const* lower, const thc_opts* opts,
                                    double* energies, thc_mps* state, const thc_allocator* alloc,
                                    void* stream);

/* One global-Krylov time step (Sec. 2.2, Eq. Krylov_combination): K Krylov
 * vectors v_i from psi/|psi| (Gram-Schmidt by mps_add_compress, as
 * krylov_lanczos_ground), the projected Htil and S, the correction of
 * Eq. reortho / Eq. eff_H by canonical orthogonalisation, and
 * a(dt) = exp(-i dt Heff) a(0) in the orthonormalised basis (a complex
 * Hermitian float64 eigensolver on the device); then
 * psi(dt) = compress(sum_i |psi| a_i v_i) by the pairwise reduction,
 * renormalised to |psi|.  psi: real or complex MPS of the path's precision
 * (a real psi is converted to complex first), bonds at most
 * min(D_max, 4^b, 4^(L-b)); D_max <= 256.  lost_norm (host, may be NULL) =
 * 1 - |psi(dt)|/|psi| before the renormalisation.  `out` receives a
 * library-owned complex MPS (C128 for path FP64, C64 for FP32).
 * Errors: THC_EINVAL (bad input, dt not finite), THC_EUNSUPPORTED (bonds or
 * D_max out of range), THC_EBREAKDOWN (psi = 0), THC_ETIMEOUT (the small
 * eigensolver ran out of sweeps). */
thc_status krylov_expm_apply(const thc_hamiltonian* H, const thc_mps* psi, double dt, int K,
                             const thc_opts* opts, thc_mps* out, double* lost_norm,
                             const thc_allocator* alloc, void* stream);

/* The adjoint of the THC-MPO expectation value: E = <phi|H|psi> for H of Eq. 1
 * with v of Eq. thc, contracted exactly (no compression) term by term through
 * the bond-2 ladder MPOs of Sec. 3.1 (the 4N^2 Coulomb terms G_{mu s, nu s'} of
 * Eq. G and the one-body terms (sum_p t_pq a+_{p s}) a_{q s}), with left and
 * right environments; the derivatives are the reverse-mode contractions of
 * the same networks (the paper computes no derivatives; this serves
 * differentiation through H's factors and the state).
 *  - phi, psi: real MPS (F64 on path FP64, F32 on FP32 / TF32), equal L, any
 *    bonds up to 4096 (memory permitting).
 *  - value: host double, E.
 *  - grad_t [L*L], grad_chi [L*N], grad_zeta [N*N]: device float64, row-major
 *    like t, chi, zeta; written with dE/dt_pq, dE/dchi^mu_p, dE/dzeta^{mu nu}
 *    (every entry an independent variable); each may be NULL.
 *  - grad_psi: optional output MPS (psi's bonds and dtype), site i =
 *    dE/d(site i of psi); NULL to skip.
 *  - opts: path, batch (terms in flight) and the term range (thc_apply_H's
 *    term indexing; the value and derivatives are then those of the sum of
 *    the terms in range) are used; D_max and tol are not (nothing is
 *    truncated).
 * Errors: THC_EINVAL, THC_EUNSUPPORTED (complex MPS), THC_ENOMEM, THC_ECUDA. */
thc_status thc_expect_grad(const thc_hamiltonian* H, const thc_mps* phi, const thc_mps* psi,
                           const thc_opts* opts, double* value, double* grad_t, double* grad_chi,
                           double* grad_zeta, thc_mps* grad_psi, const thc_allocator* alloc, void* stream);

/* Eigen-decomposition t = U diag(lambda) U^T of the one-body integrals (App. D,
 * Eq. t_diagonalization) by a float64 Jacobi kernel: t device [L*L] row-major,
 * lambda device [L] ascending, u device [L*L] row-major with column i the
 * eigenvector of lambda_i. */
thc_status thc_kinetic_factors(int L, const double* t, double* lambda, double* u, void* stream);

/* Release a library-owned MPS (owner != NULL) and clear the descriptor. */
void thc_mps_free(thc_mps* m, const thc_allocator* alloc, void* stream);

/* Message for the last non-OK status returned on the calling thread. */
const char* thc_last_error(void);

/* Build description (arch, compiler) as a static string. */
const char* thc_build_info(void);

/* Diagnostics (no counterpart in the paper).  thc_kernel_launches: number of
 * CUDA kernels this library has launched in the process so far.
 * thc_profile_enable(1) makes every later launch record a pair of CUDA events
 * on its own stream; thc_profile_read synchronises those events, writes a JSON
 * object {"name": {"launches": n, "ms": total}, ...} of the per-kernel sums
 * since the last read into buf (NUL-terminated, truncated to len), resets the
 * sums, and returns the number of bytes the full text needs.  The entry
 * "jacobi_budget_exhausted" counts Jacobi SVDs that used their whole sweep
 * budget ("ms" then holds the most rotations a last sweep still applied); with
 * profiling on,
 * "jacobi_sweeps_all" / "jacobi_sweeps_p_ge_128" count the Jacobi SVDs
 * ("launches") and their sweeps ("ms" holds the sweep total).  Profiling adds
 * host work per launch; leave it off for timed runs. */
unsigned long long thc_kernel_launches(void);
void thc_profile_enable(int on);
int thc_profile_read(char* buf, int len);

/* <phi|psi> (float64 accumulation, as mps_inner) for callers that cannot
 * allocate GPU memory -- e.g. code running inside a framework whose memory
 * pool forbids foreign allocations, real-time loops that must not touch an
 * allocator, or embedders with a memory budget fixed up front.  The paper has
 * no counterpart; this is a deployment variant of mps_inner.
 *  - Allocates nothing: the scratch (the float64 transfer matrices) is one
 *    file-scope device array of 16 MiB.  It is reserved on a device when the
 *    library's module is first used there (lazy module loading, the CUDA
 *    default) and held until the process exits.  phi and psi are read in
 *    place; real MPS only (F64 or F32), with the limits of mps_inner (equal L
 *    in [2, 64], d = 4, bonds in [1, 4096]).
 *  - Limit: 8 * (chi_phi * chi_psi * 5 + 64) bytes (rounded) must fit in
 *    16 MiB, i.e. max bond products up to about 4e5 (512 x 512 works); larger
 *    inputs return THC_EINVAL and nothing is launched.
 *  - The first call on a device looks up the array's device address with that
 *    device current.  The call reads its result back to the host and
 *    synchronises `stream`, so it must not be made while `stream` is being
 *    captured into a CUDA graph: such a call returns THC_EUNSUPPORTED and
 *    enqueues nothing.
 *  - All calls share the array and it keeps the previous call's contents (the
 *    kernels initialise what they read).  Calls whose GPU work overlaps (other
 *    streams without ordering, other threads) race on it.
 *  - out_re: host pointer; the call synchronises `stream` before returning.
 *    Errors: THC_EINVAL (bad or oversize input), THC_EUNSUPPORTED (stream under
 *    capture), THC_ECUDA; see thc_last_error(). */
thc_status mps_inner_noalloc(const thc_mps* phi, const thc_mps* psi, double* out_re, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* THC_H */
