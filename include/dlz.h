/*
 * dlz -- deflated restarted Lanczos solvers for the hermitian Wilson-Dirac
 * operators on one GB300 GPU (sm_103a).  C ABI.
 *
 * Method: A. M. Abdel-Rehim, R. B. Morgan, D. A. Nicely, W. Wilcox,
 * "Deflated Hermitian Lanczos Methods for Multiple Right-Hand Sides"
 * (arXiv:0901.3163).  The first right-hand side is solved by Lan-DR(m,k)
 * on D^dagger D (Sec. 1: CG implementation of Lanczos, optimal for positive
 * definite spectra) or MinRes-DR(m,k) on Q = gamma5 D (Sec. 1: MinRes
 * implementation, optimal for indefinite spectra); both keep k
 * eigenvectors across restarts and return them.  Later right-hand sides
 * are solved by D-CG / D-MinRes: a Galerkin projection over the k vectors
 * at the start, then CG / MinRes (Sec. 2).
 *
 * Conventions shared with every caller:
 *   lattice dims[4] = {Lx, Ly, Lz, Lt}; V = Lx*Ly*Lz*Lt;
 *   site s = ((t*Lz + z)*Ly + y)*Lx + x (x fastest);
 *   spinor: V x 4 spins x 3 colours complex, component a = 3*spin + colour,
 *           interleaved re/im, i.e. complex128 [V][4][3] (n = 12 V);
 *   gauge:  4 directions (x, y, z, t) x V links, each a row-major 3x3
 *           complex128 matrix: [4][V][3][3], U[mu][s] links s to s + mu;
 *   D psi(x) = psi(x) - kappa sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                    + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)]
 *   with the chiral gamma basis (gamma_k = [[0,-i sigma_k],[i sigma_k,0]],
 *   gamma_4 = [[0,1],[1,0]], gamma5 = diag(1,1,-1,-1)), periodic boundaries
 *   and optionally antiperiodic time (bc_t = -1).  Sec. 2 calls D "M".
 *
 * Memory: every vector argument is a plain pointer that may be device
 * memory or host memory (pageable or pinned); the library detects which
 * (cudaPointerGetAttributes) and copies host data in and out itself.  The
 * caller owns all vector memory.  Objects (dlz_op_t, dlz_defl_t) are owned
 * by the library and released with their destroy call.  All GPU work is
 * ordered on the stream given to dlz_create_operator (0 = legacy default
 * stream); the solver calls return when their results are complete.
 *
 * Errors: every call returns DLZ_OK (0) or a negative DLZ_ERR_* code; no
 * C++ exception crosses the ABI.  dlz_strerror() names a code,
 * dlz_last_error() gives the message of the last failure on this thread.
 *
 * Environment (read at the call; none changes a result beyond the rounding of block
 * sums, apart from DLZ_WAIT_LIMIT's error path):
 *   DLZ_NO_GRAPHS=1   launch kernels one by one instead of replaying CUDA graphs
 *                     (read when an operator is created);
 *   DLZ_TRACE=1       per-cycle and per-phase timing lines on stderr;
 *   DLZ_MULTI_TILE=1|2|4  fix the block tile of dlz_batch_dminres (chunks of 128
 *                     sites per block or per work item) instead of choosing it by
 *                     timing; every tile gives the same bits;
 *   DLZ_MULTI_FORM=graph|persistent  fix the launch form of dlz_batch_dminres
 *                     (see dlz_batch_last_choice); both forms give the same bits;
 *   DLZ_WAIT_LIMIT=n  polls before a grid-barrier wait of the persistent form gives up
 *                     (default 2^24, about a second); a test hook for the timeout path;
 *   DLZ_SLAB=n        z-planes per slab of the block walk of the batched FP32 stencils
 *                     (default: the largest divisor of Lz whose slab's traffic fits in
 *                     36 MB; Lz is the plain site order); the block sums, and so the
 *                     rounding, follow the blocks;
 *   DLZ_CG_STAGE=1    the fused CGNR kernels copy their gather ranges into shared
 *                     memory first (bulk asynchronous copies); same bits as the default,
 *                     which reads the neighbours from global memory and is faster.
 */
#ifndef DLZ_H
#define DLZ_H

#ifdef __cplusplus
extern "C" {
#endif

#define DLZ_OK 0
#define DLZ_ERR_BADARG (-1)         /* invalid argument (null, size, enum)        */
#define DLZ_ERR_BAD_GAUGE (-2)      /* gauge field not SU(3) to 1e-10 or not finite */
#define DLZ_ERR_NONFINITE (-3)      /* NaN/Inf met in an input or a reduction      */
#define DLZ_ERR_NOT_CONVERGED (-4)  /* iteration limit hit; outputs hold the last iterate */
#define DLZ_ERR_BREAKDOWN (-5)      /* Lanczos breakdown (invariant subspace)       */
#define DLZ_ERR_DEVICE_TIMEOUT (-6) /* a bounded device wait gave up                */
#define DLZ_ERR_CUDA (-7)           /* CUDA runtime error                           */
#define DLZ_ERR_OOM (-8)            /* device allocation failed                     */
#define DLZ_ERR_IO (-9)             /* file read/write failed or bad file           */

/* Operators (Sec. 2): D (the Wilson matrix M), D^dagger, Q = gamma5 D, D^dagger D. */
#define DLZ_D 0
#define DLZ_DDAG 1
#define DLZ_Q 2
#define DLZ_DDAGD 3

/* Arithmetic of the hot loop. */
#define DLZ_F64 0   /* plain FP64 everywhere                                     */
#define DLZ_F32 1   /* FP32 stencil and Krylov vectors inside an FP64 defect-correction
                       loop (FP64 x, residual and deflation projection)           */
#define DLZ_BF16 2  /* dlz_apply / dlz_stencil_bench only: complex64 user vectors
                       stored as bfloat16 inside (rounded to nearest even), FP32
                       arithmetic, result rounded to bfloat16 once               */

typedef struct dlz_op_s *dlz_op_t;
typedef struct dlz_defl_s *dlz_defl_t;
typedef struct dlz_net_s *dlz_net_t;

/* Solver parameters; dlz_params_default() fills the defaults given here. */
typedef struct {
    int m;               /* Krylov dimension per cycle (Lan-DR(m,k), MinRes-DR(m,k)); 40 */
    int k;               /* eigenvectors kept across restarts; 10                        */
    double tol;          /* stop on ||b - D x|| / ||b|| <= tol (Sec. 2 residual of M^-1); 1e-10 */
    double tol_eig;      /* kept Ritz residuals must reach this (<= 0: 1e-10 * ||A|| est.); 0 */
    double oversolve;    /* extra MVPs after linear convergence, as a fraction of the
                            MVPs before it (Sec. 2: at most a factor of two); 1.0         */
    int max_cycles;      /* restart cycles (DR solvers); 1000                            */
    int max_iter;        /* iterations (D-CG / D-MinRes); 100000                         */
    int reorth_period;   /* MinRes-DR: re-orthogonalise against the kept vectors every
                            this many Lanczos steps, at the restart vector and the first
                            new step (Sec. 2: periodic, period not given); Lan-DR does it
                            at every step when this is > 0 (its converged regular Ritz
                            vectors need it); 0 turns it off; 10                          */
    int precision;       /* DLZ_F64 or DLZ_F32 (hot loop of D-CG / D-MinRes); DLZ_F64     */
    double reliable_delta; /* DLZ_F32: each FP32 inner solve reduces the residual by
                              this factor, then x is updated, the residual recomputed
                              in FP64 and projected over the deflation set again (defect
                              correction); 1e-2 (on the 16^3x32 workload 6444 D-MinRes
                              iterations against 9540 with 1e-5: the re-projection
                              removes the deflated directions FP32 lets back in).
                              D-CG holds it at 2e-3 or more (its inner solve tracks the
                              residual norm by a recurrence that levels off near 3e-4) */
    int check_every;     /* D-CG / D-MinRes: read the residual on the host every this
                            many iterations; 16                                          */
    int profile;         /* 1: time every stencil launch with CUDA events (stats)  ; 0   */
    int finish;          /* DR solvers, DLZ_F64: when the restart cycles end before the
                            residual reaches tol (max_cycles), finish the solve with
                            D-MinRes / D-CG from the current x over the deflation set
                            just built (1) or return DLZ_ERR_NOT_CONVERGED (0).  The
                            DLZ_F32 form always finishes this way; 0                     */
    int eig_only;        /* DR solvers: 1 runs Lan-DR / MinRes-DR as an eigensolver (the
                            use Sec. 2 describes for the kept eigenvectors, and the paper's
                            k = 150 study): the cycles stop as soon as every kept Ritz
                            residual is <= tol_eig (<= 0: 1e-10 ||A|| est. in FP64,
                            1e-5 ||A|| in FP32), whatever the linear residual; x is still
                            the cycles' iterate and no finishing solve runs.
                            stats.converged = 1 when the kept pairs converged, and the
                            call returns DLZ_ERR_NOT_CONVERGED when max_cycles ran out
                            first; 0                                                     */
} dlz_params;

/* Per-solve statistics. */
typedef struct {
    int converged;          /* 1 if ||b - D x|| / ||b|| <= tol was verified in FP64   */
    int iterations;         /* CG / MinRes iterations, or Lanczos steps               */
    int cycles;             /* restart cycles (DR solvers)                            */
    long long mvps;         /* applications of D or D^dagger (D^dagger D counts 2)     */
    double true_residual;   /* ||b - D x|| / ||b|| recomputed in FP64 at exit          */
    double seconds;         /* wall time of the call                                  */
    double stencil_ms;      /* profile = 1: summed device time (CUDA events) of the stencil
                               launches in the hot-loop precision (FP32 for DLZ_F32)   */
    long long stencil_launches; /* profile = 1: number of those launches                */
    double stencil_bytes;   /* profile = 1: their algorithmic bytes: per site 48 reals per
                               right-hand side (spinor in and out) + 4 links (72 reals
                               in FP64; 48 in FP32, which stores two rows per link)    */
    long long gpu_launches; /* kernels launched by this call                          */
    double kernel_ms[3];    /* profile = 1: the timed stencil launches split by kernel kind:
                               [0] plain stencil launches, [1] the first fused stencil
                               kernel of the inner solver (k_cg_k1, k_minres_k1,
                               k_lanczos_k1), [2] the second (k_cg_k23); device ms      */
    double kernel_bytes[3]; /* their algorithmic bytes (spinor reals of the fused kernel's
                               reads and writes per site and right-hand side + links)  */
    long long kernel_launches[3]; /* their launch counts                                 */
} dlz_stats;

/* Fills *p with the defaults listed above (library interface; no counterpart in the
 * paper, which fixes m, k and the tolerance per experiment in Sec. 1-2). */
int dlz_params_default(dlz_params *p);

/* Name of an error code; static storage (library interface; no counterpart in the
 * paper). */
const char *dlz_strerror(int code);
/* Message of the last failing call on this thread; static per-thread storage (library
 * interface; no counterpart in the paper). */
const char *dlz_last_error(void);

/*
 * Creates the Wilson operator D for the gauge field `gauge` (complex128
 * [4][V][3][3], host or device) with hopping parameter kappa (Sec. 2) and
 * time boundary bc_t (+1 periodic, -1 antiperiodic).  The library keeps its
 * own FP64 and FP32 copies of the links in its internal layout.  Every link
 * is checked to be SU(3) to 1e-10 (||U^dag U - 1||_max, |det U - 1|):
 * DLZ_ERR_BAD_GAUGE otherwise.  `stream` is a cudaStream_t (may be 0).
 * dims[i] >= 1; V * 12 must fit in a 32-bit signed int.
 */
int dlz_create_operator(const int dims[4], const void *gauge, double kappa, int bc_t,
                        void *stream, dlz_op_t *out);
/* Releases an operator and its device memory (library interface; no counterpart in the
 * paper).  Deflation sets made on it must be destroyed first. */
int dlz_destroy_operator(dlz_op_t op);
/* Lattice volume V of the operator: the sites of the Wilson matrix of Sec. 2 (V/2 for
 * an even-odd operator). */
int dlz_op_volume(dlz_op_t op, long long *V);

/*
 * Even-odd (Schur complement) operator -- not in the paper: the standard reduction
 * of D x = b to the even sites (x + y + z + t even), to which Lan-DR, MinRes-DR,
 * D-CG and D-MinRes apply unchanged.  The hopping term of D = 1 - kappa H links
 * only sites of opposite parity, so D x = b is
 *   Dhat x_e = b_e + kappa H_eo b_o,  Dhat = 1 - kappa^2 H_eo H_oe,
 *   x_o = b_o + kappa H_oe x_e,
 * and Dhat^dag = gamma5 Dhat gamma5, so Qhat = gamma5 Dhat is hermitian.
 * dlz_create_operator_eo: arguments as dlz_create_operator; every extent must be
 *   even.  The operator's vectors are even-site spinors, complex128 [V/2][4][3]
 *   holding the even sites in increasing site order; dlz_op_volume gives V/2.  On it
 *   DLZ_D / DLZ_DDAG / DLZ_Q / DLZ_DDAGD mean Dhat, Dhat^dag, Qhat, Dhat^dag Dhat in
 *   dlz_apply, dlz_apply_noalloc and dlz_stencil_bench (DLZ_F64, DLZ_F32), and
 *   dlz_landr / dlz_minresdr / dlz_dcg / dlz_dminres solve Dhat x_e = b_e with the
 *   same meaning of every parameter (the stopping residual is ||b_e - Dhat x_e|| /
 *   ||b_e||).  Not built for it: bfloat16 storage, FP32 D-MinRes (DLZ_F64 D-MinRes
 *   and FP32 / FP64 D-CG are), dlz_batch_dminres and the network (DLZ_ERR_BADARG).
 *   Deflation files record the operator kind and load only into the same kind.
 *   The operator holds two odd-site work fields of 16 right-hand sides (FP64 and
 *   FP32), allocated at creation.
 * dlz_eo_prepare: b (complex128 [nrhs][V][4][3], host or device) -> b_e =
 *   even part of b + kappa H_eo (odd part of b), complex128 [nrhs][V/2][4][3].
 * dlz_eo_reconstruct: x = (x_e, b_o + kappa H_oe x_e) in the full layout
 *   [nrhs][V][4][3], from x_e [nrhs][V/2][4][3] and the same b.
 * ||b - D x|| = ||b_e' - Dhat x_e|| for b_e' = dlz_eo_prepare(b): the odd rows of
 * D x = b hold exactly, so the full residual is the even-site residual.
 */
int dlz_create_operator_eo(const int dims[4], const void *gauge, double kappa, int bc_t,
                           void *stream, dlz_op_t *out);
int dlz_eo_prepare(dlz_op_t op, const void *b, void *b_e, int nrhs);
int dlz_eo_reconstruct(dlz_op_t op, const void *x_e, const void *b, void *x, int nrhs);

/*
 * out = A in for A = DLZ_D, DLZ_DDAG, DLZ_Q or DLZ_DDAGD (Sec. 2: M, M^dagger,
 * gamma5 M, M^dagger M), on `nrhs` spinors stored one after another.
 * dtype DLZ_F64: complex128 [nrhs][V][4][3]; DLZ_F32: complex64, computed in
 * FP32; DLZ_BF16: complex64 in and out, stored as bfloat16 inside (in rounded
 * once, FP32 arithmetic, out rounded once; D^dag D rounds its intermediate
 * gamma5 D too).  in and out must not overlap.  nrhs = 0 is a no-op.
 */
int dlz_apply(dlz_op_t op, int which, const void *in, void *out, int dtype, int nrhs);

/* Size of the library's static device scratch used by dlz_apply_noalloc. */
#define DLZ_NOALLOC_SCRATCH_BYTES (64u << 20)

/*
 * dlz_apply without any device allocation (the paper has no counterpart: it
 * is a library-interface variant of dlz_apply).  For callers that cannot
 * allocate device memory at the point of the call: a caller whose memory pool
 * already holds the device's free memory (cudaMalloc would fail), or one that
 * keeps other streams busy and cannot afford the device-wide synchronisation
 * of the cudaFree that dlz_apply's temporary buffers end with.
 *
 * Same operation, arguments and layout as dlz_apply (dtype DLZ_F64 or DLZ_F32
 * only), except: in and out must
 * be device (or managed) pointers (host pointers: DLZ_ERR_BADARG, since
 * staging them would allocate), and the packed work vectors live in one
 * static device array of DLZ_NOALLOC_SCRATCH_BYTES per device: 2 vectors of
 * 12 V complex values (3 for DLZ_DDAGD), 16 B per value for DLZ_F64 and 8 B
 * for DLZ_F32.  Lattices that need more are rejected with DLZ_ERR_BADARG
 * before any work is queued (16^3x32: every case fits except DLZ_F64 with
 * DLZ_DDAGD).  Nothing in the scratch has to start at zero: every element is
 * written before it is read.
 *
 * The array is shared by every operator and thread of the process on that
 * device: two calls that overlap in time (different host threads, or
 * operators on different streams) race on it and give wrong results; the
 * caller must serialise them.  The call is synchronous (returns after the
 * operator's stream has finished the work), like dlz_apply.  The first call
 * on each device looks the array's address up (cudaGetSymbolAddress) and
 * should come before any stream capture that the caller starts.  Returns
 * DLZ_ERR_CUDA if that lookup fails.  The address is kept per device for
 * the life of the process: after a cudaDeviceReset (a new context, where the
 * array may sit elsewhere) the kept address is stale, so a process that resets
 * a device must not call dlz_apply_noalloc on it again.
 *
 * The array is part of the library's device code: every process that loads
 * the library holds DLZ_NOALLOC_SCRATCH_BYTES on each device it uses, whether
 * or not it ever calls dlz_apply_noalloc, until the process exits.
 */
int dlz_apply_noalloc(dlz_op_t op, int which, const void *in, void *out, int dtype, int nrhs);

/*
 * Lan-DR(m,k) on A = D^dagger D for D x = b (Sec. 1, Sec. 2): solves
 * D^dagger D x = D^dagger b by restarted Lanczos with a Galerkin solve per
 * cycle, keeping the k lowest regular Ritz vectors across restarts, and
 * runs past linear convergence until the kept Ritz residuals reach tol_eig
 * (or the oversolve budget is spent).  b, x: complex128 [V][4][3] (x is
 * output only; the start vector is 0).  If defl_out is not NULL it receives
 * the deflation set (k vectors + H = V_k^dag A V_k) for dlz_dcg.
 * Returns DLZ_ERR_NOT_CONVERGED (x and defl still valid) if max_cycles ran out.
 */
int dlz_landr(dlz_op_t op, const void *b, void *x, const dlz_params *p,
              dlz_defl_t *defl_out, dlz_stats *stats);

/*
 * MinRes-DR(m,k) on Q = gamma5 D for D x = b (Sec. 1, Sec. 2): solves
 * Q x = gamma5 b by restarted Lanczos with a least-squares (minimum residual)
 * solve per cycle, keeping k harmonic Ritz vectors (nearest zero) across
 * restarts.  Arguments and returns as dlz_landr; the deflation set is for
 * dlz_dminres.
 */
int dlz_minresdr(dlz_op_t op, const void *b, void *x, const dlz_params *p,
                 dlz_defl_t *defl_out, dlz_stats *stats);

/*
 * D-CG (Sec. 2): for each of the nrhs right-hand sides B[i] (complex128
 * [nrhs][V][4][3]) the Galerkin projection x0 = V_k H^-1 V_k^dag D^dag b over
 * the deflation set, then CG on D^dagger D x = D^dagger b, stopping on the
 * FP64-verified ||b - D x|| / ||b|| <= tol.  defl may be NULL (plain CG on
 * the normal equations).  stats: array of nrhs entries or NULL.  In DLZ_F32
 * the right-hand sides are solved in batches of up to 16; the time, launch and
 * profile fields of a batch's entries are the batch's totals shared out over
 * its right-hand sides (counts split so that they add up to the totals), while
 * converged, iterations, mvps and true_residual are each right-hand side's own.
 * Returns DLZ_ERR_NOT_CONVERGED if any right-hand side missed tol within max_iter.
 */
int dlz_dcg(dlz_op_t op, dlz_defl_t defl, const void *B, void *X, int nrhs,
            const dlz_params *p, dlz_stats *stats);

/*
 * D-MinRes (Sec. 2): projection x0 = V_k H^-1 V_k^dag gamma5 b over the
 * deflation set (H = V_k^dag Q V_k), then MinRes on Q x = gamma5 b.
 * Arguments as dlz_dcg; defl NULL gives plain MinRes.
 */
int dlz_dminres(dlz_op_t op, dlz_defl_t defl, const void *B, void *X, int nrhs,
                const dlz_params *p, dlz_stats *stats);

/*
 * GMRES-DR(m,k) and D-GMRES(m) on D itself (non-hermitian), FP64 only
 * (p->precision must be DLZ_F64) -- the deflated methods for non-hermitian systems
 * that the paper contrasts its hermitian methods with (its refs. [1], [2]):
 * dlz_gmresdr: restarted Arnoldi (Gram-Schmidt twice) with a least-squares solve per
 *   cycle, keeping the k harmonic Ritz vectors of smallest |theta| (eigenpairs of
 *   H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^H) across restarts; stops on the FP64
 *   ||b - D x|| / ||b|| <= tol (checked once per cycle).  Arguments as dlz_landr; the
 *   deflation set (which = DLZ_D) holds V_{k+1} and Hbar_k with D V_k = V_{k+1} Hbar_k,
 *   and its pairs are the kept harmonic Ritz pairs: dlz_defl_get gives Re theta and the
 *   FP64 residual ||D y - theta y||, dlz_defl_value_complex gives theta.  Not saved to
 *   files (dlz_defl_save: DLZ_ERR_BADARG).
 * dlz_dgmres: for each right-hand side, a minimum-residual projection over span(V_k)
 *   (y = argmin ||V_{k+1}^H r - Hbar_k y||, x += V_k y) then one GMRES(m) cycle, repeated
 *   until tol; p->max_iter bounds the Arnoldi steps.  defl NULL: plain GMRES(m).
 *   Arguments as dlz_dcg; defl must come from dlz_gmresdr on the same operator.
 */
int dlz_gmresdr(dlz_op_t op, const void *b, void *x, const dlz_params *p, dlz_defl_t *defl_out, dlz_stats *stats);
int dlz_dgmres(dlz_op_t op, dlz_defl_t defl, const void *B, void *X, int nrhs, const dlz_params *p,
               dlz_stats *stats);
/* The i-th value of a deflation set as a complex number: theta_i of a GMRES-DR set
 * (the paper's refs. [1], [2]), (value_i, 0) of the hermitian sets (Sec. 2). */
int dlz_defl_value_complex(dlz_defl_t d, int i, double *re, double *im);

/* Number k of vectors in a deflation set -- the eigenvectors the first right-hand
 * side computes and hands to the later ones (Sec. 2) -- and which operator it deflates
 * (DLZ_DDAGD from dlz_landr, DLZ_Q from dlz_minresdr, DLZ_D from dlz_gmresdr). */
int dlz_defl_count(dlz_defl_t d, int *k, int *which);
/*
 * i-th Rayleigh-Ritz pair of the deflation set (Sec. 2: the eigenvectors computed
 * while solving the first right-hand side): eigenvalues of H in ascending order, the unit vector y_i = V_k z_i (complex128 [V][4][3], host
 * or device; NULL to skip), its value y_i^dag A y_i and its residual
 * ||A y_i - value y_i|| (either pointer may be NULL).  The residuals of all k
 * pairs are computed in FP64 on the first request for one (k MVPs).
 */
int dlz_defl_get(dlz_defl_t d, int i, void *vec_out, double *value, double *residual);
/* Writes the deflation set (header, H, V_k in FP64) to a file / reads it back
 * for the same operator geometry, so that the eigenvectors of Sec. 2 outlive the
 * process (a checkpoint; no counterpart in the paper).  DLZ_ERR_IO on failure.
 * dlz_defl_destroy releases a set. */
int dlz_defl_save(dlz_defl_t d, const char *path);
int dlz_defl_load(dlz_op_t op, const char *path, dlz_defl_t *out);
int dlz_defl_destroy(dlz_defl_t d);

/*
 * D-MinRes on many lattices at once (Sec. 2's D-MinRes applied to each
 * lattice; the batching across lattices of uneven size has no counterpart in
 * the paper).  ops[l]: the operator of lattice l; defls[l]: its MinRes-DR
 * deflation set or NULL (defls itself may be NULL); B[l], X[l]: nrhs[l] <= 16
 * complex128 vectors [nrhs[l]][V_l][4][3] (host or device).  With
 * p->precision == DLZ_F32 every (lattice, right-hand side) pair is a slot of one
 * fused FP32 MinRes whose kernels cover all slots in one launch per stage
 * (a block table maps each block to its slot; CUDA-graph groups of 6
 * iterations), inside a lattice-by-lattice FP64 defect correction with the
 * Galerkin projection at every restart; the kernels run on ops[0]'s stream and
 * the per-lattice work on each operator's stream (synchronised between the two).
 * DLZ_F64: the lattices are solved one after another by dlz_dminres.
 * stats: one entry per slot, lattice-major.  Returns DLZ_ERR_NOT_CONVERGED if
 * any slot did not reach p->tol within p->max_iter inner iterations.
 */
int dlz_batch_dminres(int nlat, dlz_op_t *ops, dlz_defl_t *defls, const void *const *B, void *const *X,
                      const int *nrhs, const dlz_params *p, dlz_stats *stats);

/*
 * Products of FP32 basis vectors on the tensor cores (tcgen05, FP32 data split into
 * two TF32 parts, hi*hi + hi*lo + lo*hi accumulated in FP32): the kernels behind the
 * Rayleigh-Ritz restart V_{k+1} = V_{m+1} P of the FP32 DR solvers and the batched
 * Galerkin projection of the FP32 D-CG / D-MinRes (Sec. 1-2), exported for testing and
 * measurement.  All vector pointers are device pointers to float data; work runs on the
 * legacy default stream and the calls return when it is complete.
 * dlz_basis_combine: out[j][t] = sum_i c_ij V[i][t] for t < len floats, j < nout <= 256;
 *   V[i] at V + i * ldv, out[j] at out + j * ldo (len, ldv, ldo multiples of 4).
 *   cplx = 0: coef real, host double [nin][nout]; cplx = 1: the vectors are complex
 *   (interleaved re/im floats) and coef complex, host double [nin][nout][2].
 * dlz_basis_dots: C[q][i] = <V_i, R_q> = sum_t conj(V_i[t]) R_q[t] over the len / 2
 *   complex entries; nin <= 128, nq <= 16, len a multiple of 32; C: host complex
 *   double [nq][nin][2].  Per block, 2048 floats are summed in FP32 by the tensor
 *   cores, then in FP64.
 * Both return DLZ_ERR_BADARG for shapes outside these limits and
 * DLZ_ERR_DEVICE_TIMEOUT if a bounded wait in the kernel gave up.
 */
int dlz_basis_combine(const float *V, long long ldv, int nin, long long len, const double *coef, int nout,
                      int cplx, float *out, long long ldo);
int dlz_basis_dots(const float *V, long long ldv, int nin, const float *R, long long ldr, int nq,
                   long long len, double *C);

/*
 * (Measurement of the uneven multi-lattice batch; no counterpart in the paper.)
 * The launch form the autotuner of the last DLZ_F32 dlz_batch_dminres call chose (op:
 * that call's ops[0]): form 0 = one launch per stage replayed from CUDA graphs, 1 = one
 * persistent cooperative launch over all slots and iterations (grid barriers whose waits
 * give up after a bounded number of polls, about a second, and then make the call return
 * DLZ_ERR_DEVICE_TIMEOUT); chunks_per_block: 128-site chunks per block (or per work
 * item); half_grid: 1 if the persistent grid was half the co-resident maximum.  Any
 * pointer may be NULL.  All 0 before the first call.
 */
int dlz_batch_last_choice(dlz_op_t op, int *form, int *chunks_per_block, int *half_grid);

/*
 * Measurement entry point (the paper counts cost in matrix-vector products, Sec. 2;
 * this times one): packs `nrhs` spinors `in` (dtype DLZ_F64:
 * complex128, DLZ_F32: complex64, [nrhs][V][4][3], host or device) into the
 * internal layout and launches the stencil `which` (DLZ_D, DLZ_DDAG or DLZ_Q)
 * the way the solvers do -- all nrhs right-hand sides in one launch -- `iters`
 * times back to back on the operator's stream, after 3 untimed launches.
 * *ms_per_launch receives the average device time per launch (CUDA events).
 */
int dlz_stencil_bench(dlz_op_t op, int dtype, int which, int nrhs, int iters, const void *in,
                      double *ms_per_launch);

/*
 * Learned seed for the deflation space (no counterpart in the paper, which
 * builds the deflation space with Lan-DR / MinRes-DR only): a gauge-covariant
 * parallel-transport convolution (PTC) network on the operator's lattice and
 * links.  Layer l maps widths[l] channels to widths[l+1] channels (each a
 * spinor field):
 *   out[c'](x) = sum_o sum_c W[o][c'][c] (T_o in[c])(x),
 * o = 0, +mu (1 + 2 mu), -mu (2 + 2 mu) for mu = x, y, z, t; T_0 = 1,
 * (T_+mu psi)(x) = U_mu(x) psi(x + mu), (T_-mu psi)(x) = U_mu(x - mu)^dag psi(x - mu),
 * periodic in all directions whatever the operator's time boundary; each
 * W[o][c'][c] is a complex 4x4 spin matrix (entry [4 s' + s]).  No
 * activation: the network is linear in its input.  The kernels use the
 * weights rounded to bfloat16 and compute in FP32; an FP32 master copy is
 * what the optimiser updates.  Gradients are G(z) = dL/dRe z + i dL/dIm z.
 *
 * dlz_net_create: nlayers in [1, 8], widths[0] = widths[nlayers] = 1, every
 *   width in [1, 16]; weights: complex64, the layers one after another, each
 *   [9][widths[l+1]][widths[l]][16] (host or device; copied).
 * dlz_net_bind: the links (and stream) of another operator on the same lattice
 *   are used from now on (a network is trained over many gauge fields).
 * dlz_net_forward: in, out: device complex64 [nvec][V][4][3]; keeps every
 *   layer's input for the next dlz_net_backward.
 * dlz_net_backward: grad_out = G(out) of the last forward (same nvec);
 *   adds G(W) to the gradient buffer; grad_in (may be NULL) receives G(in).
 * dlz_net_get: what = 0 master weights, 1 gradients, 2 the bfloat16 weights in
 *   use (as complex64); host_out holds dlz_net_weight_count complex64 values.
 * dlz_net_adam_step: Adam (bias-corrected) on every real and imaginary part
 *   of the master weights, then refreshes the bfloat16 copy and clears the
 *   gradients.
 * dlz_subspace_loss: per vector f_i (device complex64 [nvec][V][4][3]),
 *   loss[i] = ||(1 - V V^dag) f_i||^2 / ||f_i||^2 against the deflation set's
 *   orthonormal vectors V (host double[nvec]); grad (device complex64, may be
 *   NULL) receives grad_scale * G(f_i) with
 *   G(f_i) = 2 ((1 - V V^dag) f_i - loss[i] f_i) / ||f_i||^2 (grad_scale = 1/nvec
 *   gives the gradient of the mean loss over the nvec vectors).
 * dlz_seed_deflation: a deflation set from k device vectors (dtype DLZ_F64:
 *   complex128, DLZ_F32: complex64, [k][V][4][3]): orthonormalised (modified
 *   Gram-Schmidt twice, in FP64), then H = V^dag A V (k MVPs of A = Q or
 *   D^dag D) and its Rayleigh-Ritz pairs, usable by dlz_dcg / dlz_dminres /
 *   dlz_defl_get.  DLZ_ERR_BREAKDOWN if the vectors are linearly dependent.
 */
int dlz_net_create(dlz_op_t op, int nlayers, const int *widths, const void *weights, dlz_net_t *net);
int dlz_net_destroy(dlz_net_t net);
int dlz_net_bind(dlz_net_t net, dlz_op_t op);
int dlz_net_weight_count(dlz_net_t net, long long *count);
int dlz_net_forward(dlz_net_t net, const void *in, int nvec, void *out);
int dlz_net_backward(dlz_net_t net, const void *grad_out, int nvec, void *grad_in);
int dlz_net_get(dlz_net_t net, int what, void *host_out);
int dlz_net_set_weights(dlz_net_t net, const void *weights);
int dlz_net_zero_grad(dlz_net_t net);
int dlz_net_adam_step(dlz_net_t net, double lr, double beta1, double beta2, double eps);
int dlz_subspace_loss(dlz_defl_t defl, const void *f, int nvec, double grad_scale, double *loss, void *grad);
int dlz_seed_deflation(dlz_op_t op, int which, const void *vecs, int dtype, int k, dlz_defl_t *defl_out);

/*
 * Host-side dense helpers used by the restart of Lan-DR and MinRes-DR (Sec. 1-2; exported
 * for testing; no GPU needed).  Row-major n x n matrices.
 *   dlz_host_symeig: eigen-decomposition of a real symmetric matrix A
 *     (Householder tridiagonalisation + implicit QR with Wilkinson shifts):
 *     w[n] ascending, Z[n][n] with the eigenvector of w[j] in column j.
 *   dlz_host_sym_extremes: the smallest (lo) and largest (hi) eigenvalue of a
 *     real symmetric A (Householder tridiagonalisation + Sturm-sequence
 *     bisection to the spacing of doubles); DLZ_ERR_NONFINITE on non-finite A.
 *   dlz_host_restart_plan: the small problem at the end of one Lan-DR
 *     (harmonic = 0) or MinRes-DR (harmonic = 1) cycle, as the solvers run it
 *     (Sec. 1-2).  In: Tbar ((m+1) x m, the Lanczos matrix of the cycle: after a
 *     restart a dense leading (k+1) x k block, then the band) and c (m+1, the
 *     residual's coefficients in the basis V_{m+1}).  Out: y[m] (x += V_m y),
 *     P[(m+1) x (k+1)] (V_{k+1} <- V_{m+1} P), Tn[(m+1) x m] and cn[m+1] (Tbar
 *     and c of the next cycle), theta[k] and ritz_res[k] (the kept regular or
 *     harmonic Ritz values and residuals); *anorm becomes
 *     max(*anorm, max |eig T_m|).  Needs 2 <= m, 1 <= k < m.
 *   dlz_host_lstsq: y = argmin ||c - T y|| for T (rows x cols, rows > cols,
 *     full column rank) by Householder QR; q[rows] receives the unit
 *     vector spanning the orthogonal complement of range(T) when rows == cols + 1
 *     (may be NULL).
 */
int dlz_host_symeig(int n, const double *A, double *w, double *Z);
int dlz_host_sym_extremes(int n, const double *A, double *lo, double *hi);
int dlz_host_lstsq(int rows, int cols, const double *T, const double *c, double *y, double *q);
int dlz_host_restart_plan(int harmonic, int m, int k, const double *Tbar, const double *c, double *y, double *P,
                          double *Tn, double *cn, double *theta, double *ritz_res, double *anorm);
/*
 * Complex host helpers of GMRES-DR (the paper's refs. [1], [2]; exported for testing; no
 * GPU needed).  Complex
 * values are interleaved (re, im) doubles, matrices row-major.
 *   dlz_host_zgeev: eigenvalues w[n] and unit eigenvectors (column j of Z, n x n; Z
 *     may be NULL) of a general complex n x n matrix A (Householder Hessenberg
 *     reduction, single-shift QR to Schur form, back substitution).
 *   dlz_host_zlstsq: y = argmin ||c - A y|| for A rows x cols, rows > cols, by
 *     Householder QR; q[rows] (may be NULL; rows == cols + 1) receives the unit vector
 *     spanning range(A)^perp.
 */
int dlz_host_zgeev(int n, const double *A, double *w, double *Z);
int dlz_host_zlstsq(int rows, int cols, const double *A, const double *c, double *y, double *q);
/*
 * The Rayleigh-Ritz step of a deflation set (Sec. 2: the eigenvectors handed from the
 * first right-hand side to the others), exported for testing; no GPU needed.  H is the
 * k x k hermitian projection V^dag A V, G the Gram matrix V^dag V of a basis that is
 * orthonormal only to rounding (NULL: orthonormal), both complex interleaved row-major.
 * values[k] (ascending) and Z (k x k complex, column j for values[j]; may be NULL) solve
 * H z = value G z with z^dag G z = 1, by a Cholesky factor of G and the eigenvectors of
 * L^-1 H L^-dag.  DLZ_ERR_BREAKDOWN if G is not positive definite.
 */
int dlz_host_rayleigh_ritz(int k, const double *H, const double *G, double *values, double *Z);

#ifdef __cplusplus
}
#endif
#endif /* DLZ_H */
