/*
 * qegb.h -- C ABI of libqegb: the plane-wave Kohn-Sham operator H|psi> and
 * the block-Davidson eigensolver on one NVIDIA GB300 GPU (sm_103a).
 *
 * The paper ("Quantum ESPRESSO toward the exascale", Sec. 3.2.1) asks that
 * the domain libraries exchange data only through plain APIs with minimal
 * use of structured types; every entry point below takes plain pointers and
 * sizes.  The one struct, qe_problem, is a flat descriptor of plain fields.
 *
 * Units: lengths in bohr, energies in Rydberg, k in Cartesian bohr^-1.
 *
 * Conventions shared by every entry point
 *  - Complex arrays are interleaved (re, im) doubles.
 *  - Plane-wave order: the order returned by qe_gsphere (ascending |k+G|^2,
 *    ties by Miller index (m1, m2, m3) lexicographically).  psi, beta and
 *    every per-plane-wave array use it.
 *  - Bands are rows: a block of nbnd bands is [nbnd][npw][2] doubles.
 *  - The real-space grid is [N3][N2][N1], x (the first lattice vector)
 *    fastest; grid point r_j = sum_i (j_i / N_i) a_i.
 *  - Memory: `mem` = QE_HOST means every array pointer of the call is host
 *    memory (the library copies in and out); QE_DEVICE means every array
 *    pointer is device memory on the context's GPU and the call is ordered on
 *    `stream` (a cudaStream_t, or NULL for the legacy default stream).
 *  - Ownership: the library never keeps a caller pointer after the call
 *    returns (for QE_DEVICE, after the work queued on `stream` completes).
 *  - Errors: every call returns a QE_* status and never aborts the process;
 *    qe_last_error() gives a message for the calling thread's last failure.
 *  - Thread safety: one qe_ctx per host thread.
 */
#ifndef QEGB_H
#define QEGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  QE_OK = 0,        /* success */
  QE_EINVAL = 1,    /* invalid argument (sizes, grid too small, null pointer) */
  QE_ENOMEM = 2,    /* device or host allocation failed */
  QE_ENOCONV = 3,   /* Davidson hit max_iter: the best bands are still returned */
  QE_EAGAIN = 4,    /* serving queue full, retry later */
  QE_PENDING = 5,   /* serving: request not finished yet */
  QE_ETIMEOUT = 6,  /* a bounded device wait ran out */
  QE_ECUDA = 7,     /* a CUDA runtime call failed (message in qe_last_error) */
  QE_ECANCELED = 8  /* serving: request was cancelled */
};

enum { QE_FP64 = 0, QE_MIXED = 1 };   /* arithmetic of the GPU path */
/* Flags or-ed into `precision` (k = 0 only; Sec. 3.3 notes the Gamma-point
 * trick of real wavefunctions, which halves the FFT work):
 *  QE_GAMMA (qe_hpsi): every band is real in r, c(-G) = conj c(G); two bands
 *    share each FFT and the projections are taken real.  The result is H
 *    applied to that part of each band.  Ignored when k != 0.
 *  With qe_davidson and qe_davidson_batch, a k = 0 solve whose projectors
 *    are real in r (B_i(-G) = conj B_i(G) within 1e-12 of max |B|) can keep
 *    every basis vector real in r: the start bands are replaced by their
 *    larger real-in-r part, H runs as with QE_GAMMA, and the returned
 *    eigenvectors are real in r (same eigenvalues).  QE_GAMMA asks for it;
 *    by default solves on grids of at least 48^3 points use it (smaller FFTs
 *    gain less than the mode's extra launches cost), except QE_MIXED solves
 *    with QE_RR_FP32 (whose FP32 phase converges in fewer iterations on
 *    complex bands).
 *  QE_NO_GAMMA (qe_davidson, qe_davidson_batch): never. */
enum { QE_GAMMA = 0x100, QE_NO_GAMMA = 0x200 };
/* QE_FFT_FP64PIPE (qe_hpsi, with QE_FP64): run the FFT in float64 on the FP64
 * pipe instead of in float-float pairs on the FP32 pipes (the default; same
 * 1e-12 accuracy class, several times the throughput on GB300, whose FP64
 * rate is 1/64 of its FP32 rate).  Ignored with QE_MIXED. */
enum { QE_FFT_FP64PIPE = 0x400 };
/* QE_RR_FP32 (qe_davidson, qe_davidson_batch, with QE_MIXED): solve the
 * reduced eigenproblems of the mixed iterations (Cholesky of the overlap
 * matrix, tridiagonal eigensolver) in FP32.  By default QE_MIXED keeps the
 * Rayleigh-Ritz step in FP64 (on reduced matrices from its TF32x3 products).
 * Ignored with QE_FP64. */
enum { QE_RR_FP32 = 0x800 };
/* QE_SAME_OPERATOR (qe_hpsi, device memory): the operator -- vloc_r, beta and
 * dmat -- is the same (same pointers, same contents, same cell, k, cut-off
 * and grid) as in this context's previous qe_hpsi call at the same precision,
 * so the forms prepared from it then (the potential in the FFT's order, the
 * tensor-core slices or packs of beta) are used as they are instead of being
 * rebuilt; the caller promises that nothing changed in between (results are
 * undefined otherwise).  Quantum ESPRESSO likewise builds these once per k
 * point and applies H many times.  Without a matching previous call the flag
 * has no effect; other entry points on the context in between may clear it. */
enum { QE_SAME_OPERATOR = 0x1000 };
enum { QE_HOST = 0, QE_DEVICE = 1 };  /* where the caller's arrays live */

typedef struct qe_ctx qe_ctx;

/* Flat problem descriptor (caller-owned; read during the call only). */
typedef struct {
  double lat[9];          /* rows a1, a2, a3 (bohr) */
  double k[3];            /* k-point, Cartesian (bohr^-1) */
  double ecutwfc;         /* kinetic cut-off of the wavefunctions (Ry) */
  int grid[3];            /* FFT grid N1, N2, N3; N_i >= 2 max|m_i| + 1 */
  const double* vloc_r;   /* V_loc(r) samples [N3][N2][N1] (Ry), real */
  int nproj;              /* number of projectors (0 allowed) */
  const double* beta;     /* <k+G|beta_i>, complex [nproj][npw][2] */
  const double* dmat;     /* D_ij (Ry), real symmetric [nproj][nproj] */
  int nbnd;               /* bands in the block */
  int mem;                /* QE_HOST or QE_DEVICE, for vloc_r, beta, dmat */
} qe_problem;

/* Message for the calling thread's last failed call ("" if none). */
const char* qe_last_error(void);

/* Create a context on CUDA device `device`.  Holds a plan cache (one plan per
 * (lattice, k, cut-off, grid)) and the device workspaces.  QE_ECUDA if the
 * device cannot be used. */
int qe_ctx_create(int device, qe_ctx** out);
void qe_ctx_destroy(qe_ctx* ctx);

/* Per-kernel timing (the timing utilities of UtilXlib, Sec. 3.1).  enable=1
 * resets the counters and records a pair of CUDA events around every kernel
 * the context launches afterwards (on the launching stream); enable=0 stops
 * recording.  Launches are counted whether or not timing is on. */
int qe_profile(qe_ctx* ctx, int enable);

/* Read entry `index` (0-based, in first-launch order): kernel name (copied
 * into name[name_len]), number of timed launches and their summed device
 * time in ms.  Waits for the recorded events.  `launches` (may be NULL)
 * receives the number of kernels launched since the last reset.  index < 0
 * only reports `launches`.  QE_EINVAL past the last entry. */
int qe_profile_read(qe_ctx* ctx, int index, char* name, int name_len,
                    long long* calls, double* ms, long long* launches);

/* Test hook for the bounded device waits (failure handling of the timing and
 * error utilities, Sec. 3.1): with wait_ns > 0, every grid-wide barrier of
 * the cooperative dense-eigensolver kernels launched by this context's
 * Davidson solves waits for one arrival more than its grid supplies, for at
 * most wait_ns nanoseconds, so that each barrier runs out: the kernel sets
 * the error word and returns, and the solve returns QE_ETIMEOUT with the
 * context still usable.  wait_ns = 0 restores normal barriers (2 s limit).
 * Affects solves started after the call. */
int qe_test_grid_wait(qe_ctx* ctx, long long wait_ns);

/* Plane-wave sphere (Sec. 3.2.2 item (vi): generation of plane waves and their
 * mapping to FFT grids).  S_k = { m : |k + sum_i m_i b_i|^2 <= ecut (1 + 1e-12) },
 * b_i = 2 pi (a_j x a_k) / (a_1 . (a_2 x a_3)).  The ordering value |k+G|^2 is
 * the float64 expression ((qx*qx + qy*qy) + qz*qz) with
 * q_c = ((k_c + m1*b1_c) + m2*b2_c) + m3*b3_c, each operation rounded.
 * Host-only.  Call with miller == NULL to get the count in *npw; otherwise
 * *npw is the capacity of miller ([*npw][3] ints) and kin (optional, may be
 * NULL, [*npw] doubles |k+G|^2) and receives the count (QE_EINVAL if the
 * capacity is too small).
 * `grid` may be NULL; if given, QE_EINVAL when N_i < 2 max|m_i| + 1. */
int qe_gsphere(const double lat[9], const double k[3], double ecut,
               const int grid[3], int* npw, int* miller, double* kin);

/* Gaussian local potential sampled on the grid (the synthetic stand-in for the
 * pseudopotential's local part, Sec. 3.2.2 item (viii)):
 * V(r_j) = amp * sum_I sum_{T in {-1,0,1}^3} exp(-|r_j - R_I - T.lat|^2 / (2 sigma^2)).
 * tau: [natom][3] Cartesian positions (host).  vloc_out: [N3][N2][N1] doubles,
 * host or device per `mem`; computed on the GPU. */
int qe_vloc_gaussian(qe_ctx* ctx, const double lat[9], const int grid[3],
                     int natom, const double* tau, double amp, double sigma,
                     double* vloc_out, int mem, void* stream);

/* Kleinman-Bylander projector coefficients (Sec. 3.2.2 item (viii)) of
 * Gaussian-times-real-solid-harmonic projectors, unit L2 norm:
 * beta_{I,n,l,m}(r) = N_{n,l} S_lm(r - R_I) exp(-|r - R_I|^2 / (2 w_n^2)),
 * <k+G|beta> = Omega^-1/2 e^{-i q.R_I} N (-i)^l (2 pi)^{3/2} w^{2l+3} S_lm(q) e^{-w^2 q^2 / 2},
 * q = k + G.  Order: atom-major, then per width w_n: [s, p_x, p_y, p_z], so
 * nproj = 4 * nrad * natom.  tau [natom][3] and widths [nrad] are host arrays.
 * beta_out: complex [nproj][npw][2], host or device per `mem`; GPU-computed. */
int qe_beta_gaussian(qe_ctx* ctx, const double lat[9], const double k[3],
                     double ecut, int natom, const double* tau, int nrad,
                     const double* widths, double* beta_out, int mem,
                     void* stream);

/* H|psi> on a block of bands (Sec. 3.3: kinetic-energy, local-potential and
 * pseudopotential contributions to the Hamiltonian):
 *   (H c)_G = |k+G|^2 c_G + (1/N) sum_j e^{-iG.r_j} V(r_j) psi(r_j)
 *             + sum_ij B_i(G) D_ij sum_G' conj(B_j(G')) c_G',
 *   psi(r_j) = sum_G c_G e^{iG.r_j},  N = N1 N2 N3.
 * psi, hpsi: complex [nbnd][npw][2], host or device per prob->mem (hpsi is
 * overwritten).  precision: QE_FP64 (FP64-accurate, 1e-12 relative: FFT in
 * float-float pairs, 48-bit significand, on the FP32 pipes; projector products
 * in float64 or as Ozaki BF16 slice products on the tensor cores) or QE_MIXED
 * (FP32 FFTs and FP32 projector products, float64 in and out), optionally
 * or-ed with QE_GAMMA (k = 0: bands real in r, two per FFT) and, with
 * QE_FP64, QE_FFT_FP64PIPE.  The float-float FFT has the exponent range of
 * float: it keeps the 1e-12 accuracy for coefficients and potential values of
 * magnitude within about 1e-25 .. 1e25 (wavefunctions of any normalisation in
 * practice); outside that range use QE_FFT_FP64PIPE.
 * Errors: QE_EINVAL for bad sizes or a grid smaller than the sphere needs. */
int qe_hpsi(qe_ctx* ctx, const qe_problem* prob, int precision,
            const double* psi, double* hpsi, void* stream);

/* The same H|psi> as qe_hpsi, to the FP64 parity tolerance (1e-12 per band;
 * 2e-5 with QE_MIXED), for callers that cannot allocate device memory (no
 * counterpart in the paper).  Such callers include code running inside a
 * memory pool or arena that another component owns, under an allocator that
 * must see every allocation, or at points where a cudaMalloc would synchronise
 * the device or fail because other work holds the free memory.  qe_hpsi takes
 * its workspace from the context's buffers, which allocate on first use; this
 * entry point takes all of it from one fixed 64 MiB device array inside the
 * library (present on every GPU that loads the library, until process exit)
 * and calls no cudaMalloc, cudaFree or other allocating routine.
 *  - precision: QE_FP64 or QE_MIXED only (no QE_GAMMA, no QE_FFT_FP64PIPE:
 *    QE_EINVAL).  The FP64 projector products run on the SIMT kernels (the
 *    tensor-core slices of qe_hpsi would not fit in the array), so results
 *    differ from qe_hpsi by rounding, not bit for bit.
 *  - No context: it runs on the calling thread's current CUDA device, which
 *    must hold every array; prob->mem must be QE_DEVICE (else QE_EINVAL).
 *  - The caller passes inputs (psi, vloc_r, beta, dmat) and the output hpsi.
 *  - Size limit: the plan of the sphere, the permuted potential, the
 *    projections, one band's stick buffer and one split of the projector
 *    product must fit in 64 MiB; larger problems return QE_EINVAL with the
 *    needed size in qe_last_error() (use qe_hpsi for those).
 *  - Not callable while `stream` is being captured into a CUDA graph
 *    (QE_EINVAL): which plan the array holds is host-side state that a
 *    replayed graph would not consult.
 *  - A call whose cell, k, cut-off or grid differs from the previous call's on
 *    the device copies a new plan (the sphere's maps) from host memory into
 *    the array; that pageable copy can synchronise the calling stream.  Calls
 *    that repeat the previous problem's plan copy nothing from the host.
 *  - Every call uses the same array and leaves its contents behind; the
 *    kernels overwrite all of it that they read.  Calls whose work overlaps on
 *    the GPU (different streams, or different host threads) race on the
 *    array: order them on one stream.
 * Work is queued on `stream`; the call returns without waiting for it. */
int qe_hpsi_noalloc(const qe_problem* prob, int precision, const double* psi,
                    double* hpsi, void* stream);

/* Projectors defined instead of stored (Sec. 3.2.2 item (viii), calculation of
 * pseudopotential terms; Sec. 4 names memory per card as the bound on system
 * size).  For atom I at R_I (tau, Cartesian bohr, host) and radial function n
 * with angular momentum l[n] (0 or 1, host) and radial table
 * radial[n][G] = F_n(|k+G|) (qe_gsphere order, host or device per prob->mem):
 *   beta_{I,n,c}(G) = e^{-i (k+G).R_I} (-i)^{l_n} Y_{l_n c}(k+G) F_n(G),
 *   Y_00 = 1 / (2 sqrt(pi)),  Y_1c(q) = sqrt(3 / (4 pi)) q_c  (c = x, y, z),
 * ordered atom-major, per atom per radial function its 2 l_n + 1 components.
 * (The Gaussian projectors of qe_beta_gaussian are radial functions of each
 * width with l = 0 and l = 1 and F = Omega^-1/2 N (2 pi)^{3/2} w^{2l+3}
 * e^{-w^2 q^2 / 2}.)  At most 8 radial functions. */
typedef struct {
  int natom;
  const double* tau;      /* [natom][3] */
  int nrad;
  const int* l;           /* [nrad] */
  const double* radial;   /* [nrad][npw] */
} qe_projectors;

/* qe_hpsi with the projectors of `pj` generated on the fly: prob->beta is not
 * read (may be NULL), prob->nproj must equal natom * sum_n (2 l_n + 1) and
 * prob->dmat is D over those projectors.  The FP64 path forms beta straight
 * into the tensor-core slices of its products from per-atom phase tables (no
 * beta array is stored or copied; with host arrays none crosses the bus); the
 * other paths form the values into a work array first.  Same arguments,
 * precisions and results (to the tolerances of qe_hpsi: 1e-12 FP64, 2e-5
 * mixed) as qe_hpsi with the equivalent stored beta. */
int qe_hpsi_gen(qe_ctx* ctx, const qe_problem* prob, const qe_projectors* pj, int precision,
                const double* psi, double* hpsi, void* stream);

/* Block Davidson (Sec. 3.3, iterative solution of the Kohn-Sham Hamiltonian;
 * Sec. 3.2.1, KS_Solvers and the dense eigensolver of LAXlib) for the nbnd
 * lowest eigenpairs.  psi_inout: start bands in, Ritz vectors out
 * (complex [nbnd][npw][2]); evals [nbnd] (Ry, ascending); resid [nbnd]
 * residual 2-norms (may be NULL); iters (may be NULL) the number of basis
 * expansions.  Converged when every ||H psi_n - e_n psi_n|| <= tol.
 * max_dim: largest basis (0 selects 4 * nbnd below 64 bands, 3.5 * nbnd from 64 on).  Returns QE_ENOCONV (with the
 * best bands filled in) after max_iter expansions.  Arrays per prob->mem;
 * device work is ordered on `stream` and the call returns after it ends. */
int qe_davidson(qe_ctx* ctx, const qe_problem* prob, int precision, double tol,
                int max_iter, int max_dim, double* psi_inout, double* evals,
                double* resid, int* iters, void* stream);

/* Band-by-band conjugate-gradient eigensolver (Sec. 3.3: iterative solution of
 * the Kohn-Sham Hamiltonian with the conjugate-gradient method, beside
 * Davidson) for the nbnd lowest eigenpairs, on the same H|psi> as qe_hpsi.
 * The start bands are rotated by a Rayleigh-Ritz step; then, in a sweep, each
 * band in turn minimises its Rayleigh quotient orthogonally to the bands below
 * it along preconditioned Polak-Ribiere directions with an exact line
 * minimisation (at most max_iter iterations per band and sweep), and the sweep
 * ends with a Rayleigh-Ritz rotation of the block.  Converged when every
 * ||H psi_n - e_n psi_n|| <= tol after a rotation; QE_ENOCONV (best bands
 * filled in) after max_sweeps sweeps.  QE_MIXED sweeps with FP32 products and
 * H while residuals are above max(tol, 1e-4), then in FP64.  psi_inout, evals,
 * resid (may be NULL) as qe_davidson; iters (may be NULL): CG iterations (H
 * applications to search directions) summed over bands and sweeps.  Arrays
 * per prob->mem; device work is ordered on `stream` and the call returns after
 * it ends. */
int qe_cg(qe_ctx* ctx, const qe_problem* prob, int precision, double tol, int max_iter,
          int max_sweeps, double* psi_inout, double* evals, double* resid, int* iters,
          void* stream);

/* Charge density (Sec. 3.3: charge-density generation, on the bands of the
 * iterative solvers) of a set of bands over k points of one cell:
 *   rho(r_j) = (1 / Omega) sum_k sum_n w_nk |psi_nk(r_j)|^2,
 *   psi_nk(r_j) = sum_G c_nk(G) e^{iG.r_j},
 * on the grid [N3][N2][N1] (x fastest), Omega = |det lat|; for bands with
 * sum_G |c|^2 = 1, (Omega / N) sum_j rho(r_j) = sum_nk w_nk.
 * kpts [nk][3] (Cartesian, host); nbnd [nk] (host); psi[i]: the bands of k
 * point i, complex [nbnd[i]][npw_i][2] in that k point's qe_gsphere order;
 * weights[i]: [nbnd[i]] doubles w_nk (occupation times k weight), host arrays.
 * psi[i] and rho live per `mem` (QE_HOST / QE_DEVICE).  precision: QE_FP64
 * (FP64-accurate: the float-float FFT of qe_hpsi, sums in float64) or
 * QE_MIXED (FP32 FFT), optionally or-ed with QE_GAMMA (k = 0 points: bands
 * real in r, two per FFT).  The sum over bands and k points runs in a fixed
 * order: results are deterministic.  Device work is ordered on `stream`; with
 * QE_HOST the call returns after it ends. */
int qe_density(qe_ctx* ctx, const double lat[9], double ecut, const int grid[3], int nk,
               const double* kpts, const int* nbnd, const double* const* psi,
               const double* const* weights, int precision, double* rho, int mem, void* stream);

/* One self-consistency step of the local potential (Sec. 3.3: electronic
 * self-consistency and charge-density generation on the GPU): from the bands
 * (arguments as qe_density) the density rho, then, in Rydberg units,
 *   V_H(r)  = sum_{0 < |G|^2 <= 4 ecut} 8 pi rho~(G) / |G|^2 e^{iG.r},
 *             rho~(G) = (1/N) sum_j rho(r_j) e^{-iG.r_j}  (the density sphere),
 *   v_x(r)  = -2 (3 rho(r) / pi)^{1/3}                    (Slater exchange, LDA),
 *   V_new   = (1 - alpha) V_in + alpha (V_ext + V_H + v_x).
 * vext, vin, vnew and rho_out (optional) are [N3][N2][N1] doubles, with psi per
 * `mem`; weights are host arrays.  QE_EINVAL when the grid cannot hold the
 * density sphere (N_i < 2 max|m_i| + 1 for |G|^2 <= 4 ecut).  precision as
 * qe_density (the transforms of V_H in that arithmetic).  Device work is ordered
 * on `stream`; with QE_HOST the call returns after it ends. */
int qe_scf_step(qe_ctx* ctx, const double lat[9], double ecut, const int grid[3], int nk,
                const double* kpts, const int* nbnd, const double* const* psi,
                const double* const* weights, const double* vext, const double* vin, double alpha,
                int precision, double* vnew, double* rho_out, int mem, void* stream);

/* ---- Batches: many problems per launch --------------------------------------
 * The paper's benchmarks parallelise over k points (pools, Sec. 3.3) and note
 * that several small runs sharing one GPU pay off.  A batch applies H to the
 * bands of many problems (k points of one cell, independent cells; different
 * grids, plane-wave counts and band counts) with each FFT stage as ONE
 * persistent launch whose CTAs pull (problem, band, tile) work items from a
 * counter.  Results are bit-identical to qe_hpsi on each problem alone. */

/* H|psi> for nprob problems.  Every array of every problem (and psi[p],
 * hpsi[p], complex [probs[p].nbnd][npw_p][2]) must be device memory
 * (mem = QE_DEVICE, else QE_EINVAL).  Device work is ordered on `stream`. */
int qe_hpsi_batch(qe_ctx* ctx, int nprob, const qe_problem* probs, int precision,
                  const double* const* psi, double* const* hpsi, void* stream);

/* Block Davidson for nprob problems advanced in lockstep (k points of one
 * cell, Sec. 3.3 pools, or independent cells): every iteration applies H to
 * the new basis vectors of all unfinished solves in one batched H|psi> as
 * above.  Arguments per problem as qe_davidson (same tol, max_iter, max_dim,
 * precision for all); every array must be device memory (else QE_EINVAL).
 * status[p] (may be NULL): QE_OK, QE_ENOCONV (best bands filled in) or the
 * error of that solve; iters[p] (may be NULL) its basis expansions.  Returns
 * QE_OK when all converged, QE_ENOCONV when some did not, else the first
 * other error.  Each problem's result equals qe_davidson on it alone bit for
 * bit.  Each solve owns a workspace of the context (kept for later calls).
 * Device work is ordered on `stream`; the call returns after it ends. */
int qe_davidson_batch(qe_ctx* ctx, int nprob, const qe_problem* probs, int precision,
                      double tol, int max_iter, int max_dim, double* const* psi_inout,
                      double* const* evals, double* const* resid, int* iters, int* status,
                      void* stream);

/* A batch recorded once into a CUDA graph and replayed: qe_batch_create runs
 * the batch once (sizing and owning its own workspace), then captures its
 * launches; qe_batch_run replays them on `stream` for the SAME arrays (update
 * their contents between runs, not their addresses).  The problem descriptors
 * and the arrays they point to must stay valid while the batch exists; the
 * context must outlive it. */
typedef struct qe_batch qe_batch;
int qe_batch_create(qe_ctx* ctx, int nprob, const qe_problem* probs, int precision,
                    const double* const* psi, double* const* hpsi, void* stream,
                    qe_batch** out);
int qe_batch_run(qe_batch* batch, void* stream);
void qe_batch_destroy(qe_batch* batch);

/* Autotuner of the FFT launch shapes (sticks per CTA and threads per CTA of
 * the z and plane stages) for prob's grid at this precision: times candidate
 * shapes on the problem and keeps the fastest for every later call with that
 * grid (process-wide; also written to the file named by the environment
 * variable QE_AUTOTUNE_CACHE, read back at the next start).  Any shape gives
 * bit-identical results. */
int qe_autotune(qe_ctx* ctx, const qe_problem* prob, int precision, void* stream);

/* ---- Serving: continuous batching of Davidson solves ------------------------
 * The paper's outlook (Sec. 4) names memory per card as the bound on system size
 * and ensembles of independent runs as the way to fill large machines; Sec. 3.3
 * notes that over-subscribing one GPU with several small runs pays off.  A
 * server runs requests of different cells, cut-offs and band counts as they
 * arrive: a request is admitted, in arrival order, when one of max_slots slots
 * is idle and its estimated device footprint fits in what hbm_budget_bytes has
 * left; each slot has its own context and stream, so admitted solves overlap
 * on the GPU; a finished solve returns its workspace and the next request is
 * admitted.  Results do not depend on what else runs (kernels are
 * deterministic and each solve owns its buffers). */
typedef struct qe_srv qe_srv;

enum { QE_SERVE_FAKE_SOLVER = 1 };   /* test hook: no GPU; a solve sleeps max_iter ms */

/* max_queue: requests allowed to wait for admission (QE_EAGAIN beyond).
 * flags: 0, or QE_SERVE_FAKE_SOLVER (host-only test mode). */
int qe_serve_create(int device, size_t hbm_budget_bytes, int max_slots, int max_queue,
                    int flags, qe_srv** out);

/* Queue a Davidson solve (as qe_davidson with the default max_dim).  Every array of
 * prob and psi0 must be host memory (prob->mem = QE_HOST); they are copied
 * before the call returns.  *ticket identifies the request.  QE_EAGAIN when the
 * queue is full; QE_EINVAL when the request alone exceeds the budget. */
int qe_serve_submit(qe_srv* srv, const qe_problem* prob, int precision, double tol,
                    int max_iter, const double* psi0, uint64_t* ticket);

/* Wait up to timeout_ms (0: do not wait, < 0: wait until done) for a request.
 * QE_PENDING while it is queued or running.  When done, copies the Ritz vectors
 * (psi_out [nbnd][npw][2]), eigenvalues, residual norms, iteration count and the
 * latency from submit to completion (seconds) into the non-NULL outputs, frees
 * the request, and returns its status (QE_OK, QE_ENOCONV, QE_ECANCELED, or the
 * solve's error).  Unknown tickets: QE_EINVAL. */
int qe_serve_poll(qe_srv* srv, uint64_t ticket, int timeout_ms, double* psi_out,
                  double* evals, double* resid, int* iters, double* latency_s);

/* Cancel a request: a queued one is dropped at once, a running one finishes
 * but reports QE_ECANCELED.  QE_EINVAL for unknown tickets. */
int qe_serve_cancel(qe_srv* srv, uint64_t ticket);

/* Counters: requests submitted, completed; running now; waiting; budget bytes
 * held by running requests.  Any pointer may be NULL. */
int qe_serve_stats(qe_srv* srv, long long* submitted, long long* completed, int* running,
                   int* queued, size_t* bytes_in_use);

/* Stop: queued requests are cancelled, running ones finish, then everything is freed. */
void qe_serve_destroy(qe_srv* srv);

#ifdef __cplusplus
}
#endif
#endif /* QEGB_H */
