/*
 * pc.h -- C ABI of libpc, a GB300 (sm_103a) solver for the kernel-compensated MFD Maxwell eigenproblem of
 * photonic crystals (Jin, Xia, Xu, "Kernel compensation method for Maxwell eigenproblem in photonic crystals with
 * mimetic finite difference discretizations").
 *
 * The library computes, for Bloch vectors k, the lowest eigenpairs of the compensated operator
 *     Op = A M0 A' + gamma B'B                                            (eq. Ker_comp, Section 3.2)
 * on the periodic N^3 grid, where A = CURL_k (edges -> faces), B = DIV_k (faces -> cells) are the shifted MFD
 * operators of eq. discrete_2nd_block built from D_i = K_i + i L_i (eqs. discre, blocks), M0 = diag(1/eps) on edges
 * (Section 4.4), and gamma = 2 max{1/h, |k|^-2} (eq. pnt_number). The eigensolver is block LOBPCG (Section 5.1)
 * preconditioned by P = A A' + gamma B'B solved with FFTs (Section 5.2, Algorithm 5.1), followed by the recompute
 * check of Algorithm 4.1.
 *
 * Conventions common to every entry point
 * - Grid: N a power of two, 8 <= N <= 256, h = 1/N, on the unit cube. The cubic cell (lattice = identity) has lattice
 *   constant a = 1. A general cell (Section 2's coordinate change x = A y, Section 4.2.2) keeps the grid on the unit
 *   cube of y; D_i becomes D_hat_i = sum_j b_ji K_j + i L_i with b = A^{-1}, and the field components stay Cartesian.
 * - A face (or edge) field is complex [3][N][N][N] = (component, z, y, x), x fastest, so that D_1 acts on x.
 *   A cell field is complex [N][N][N]. A "block" of m fields stores field j at offset j * 3 N^3 (column-major
 *   tall-skinny matrix with L = 3 N^3 rows); a batch of blocks for nb k-points stores block b at offset
 *   b * stride elements.
 * - Complex numbers are interleaved (re, im): dtype PC_C128 = two doubles, PC_C64 = two floats.
 * - "device" pointers are CUDA device memory owned by the caller; "host" pointers are ordinary host memory owned by
 *   the caller. The library never frees caller memory. Pointers must be 16-byte aligned.
 * - All device work is issued on the stream given at pc_setup (or the stream argument); calls return after
 *   enqueueing unless stated otherwise. Host outputs are valid on return.
 * - Return value: 0 on success; negative on error (PC_EINVAL bad argument, PC_EUNSUPPORTED valid but not
 *   implemented, PC_ENOMEM allocation failure, PC_ECUDA CUDA error); positive warnings PC_NOT_CONVERGED and
 *   PC_SPURIOUS. pc_last_error() returns a thread-local description of the last failure.
 * - There is no CPU fallback: every numerical step runs in this library's CUDA kernels.
 */
#ifndef PC_H
#define PC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PC_OK 0
#define PC_EINVAL (-1)
#define PC_EUNSUPPORTED (-2)
#define PC_ENOMEM (-3)
#define PC_ECUDA (-4)
#define PC_NOT_CONVERGED 1
#define PC_SPURIOUS 2

#define PC_C128 0
#define PC_C64 1
#define PC_C128_DF 2 /* complex128 storage, double-float (FP32-pair) arithmetic: ~2^-44 relative rounding, FP32 pipe */

/* Preconditioner variants (Section 5.1 and Corollary discrete_vec_lap_mat). */
#define PC_PRECOND_GAMMA 0     /* P = A A' + gamma B'B, eq. penalised_marix (default) */
#define PC_PRECOND_LAPLACIAN 1 /* vector Laplacian A A' + B'B, the scalar symbol of Algorithm 5.1 */

/* Solver precision. */
#define PC_PREC_FP64 0  /* every step in FP64 / complex128 */
#define PC_PREC_MIXED 1 /* search directions in complex64; X, its residual and Gram block FP64-accurate (double-float
                           pairs on the FP32 pipe); Rayleigh-Ritz in FP64; stalled k-points finished in FP64 */

typedef struct pc_ctx pc_ctx;

typedef struct {
    int order;             /* k of Table 1: 1 (default) -> 2nd-order stencils, 2, 3, 4 -> 4th, 6th, 8th order;
                              orders above 1 need precision PC_PREC_FP64 (the mixed solve is second order) */
    double gamma_override; /* > 0: use this penalty instead of eq. pnt_number */
    int precond;           /* PC_PRECOND_GAMMA or PC_PRECOND_LAPLACIAN */
    int precision;         /* PC_PREC_FP64 or PC_PREC_MIXED */
    int guard;             /* block columns beyond nbands; < 0 (default): nbands/2 + 1, capped so 3(nbands+guard) <= 64 */
    int maxiter;           /* LOBPCG iteration cap per k-point and gamma-doubling round (default 400) */
    int max_doublings;     /* Algorithm 4.1 gamma doublings cap (default 8) */
    uint64_t seed;         /* seed of the counter-based initial blocks */
    int groups;            /* PC_PREC_MIXED: k-point groups (at most 4) iterated on separate streams so that one
                              group's latency-bound steps (Rayleigh-Ritz, host decisions) overlap the others'
                              kernels; 0 (default): 4 from 16 k-points, 2 from 8, else 1 */
    int kchunk;            /* k-points per pass of pc_solve: a batch larger than what fits the device memory (85% of
                              the free memory for the solve's panels) is solved in consecutive chunks; kchunk > 0
                              caps the chunk further; 0 (default): as many as fit */
} pc_opts;

/* Fill *opts with the defaults listed above. */
int pc_opts_default(pc_opts *opts);

/* pc_setup -- create a context for one structure (Section 4.4).
 *   out:       receives the new context (library-owned; release with pc_destroy).
 *   N:         grid points per axis (power of two, 8..256).
 *   eps_edges: host [3][N][N][N] permittivity at the edge DoFs (x-edges at ((i+1/2)h, jh, kh), etc.), all > 0.
 *              M0 = diag(1/eps_edges).
 *   lattice:   host double[9] or NULL (identity): the lattice vectors a1, a2, a3 one after the other
 *              (lattice[3 n + c] = component c of a_{n+1}), finite and linearly independent (else PC_EINVAL). The
 *              identity runs the cubic cell's kernels; any other cell runs the general-lattice stencils (every
 *              order in FP64 and complex64; second order in double-float, which the mixed solve uses). eps_edges
 *              then holds the permittivity at the Cartesian points A y of the edge midpoints y
 *              (pc_eps_spheres_lattice).
 *   opts:      options (NULL -> defaults).
 *   stream:    cudaStream_t to use for all work of this context (NULL -> the legacy default stream).
 * Uploads M0 and the FFT tables once (one host-to-device copy). */
int pc_setup(pc_ctx **out, int N, const double *eps_edges, const double *lattice, const pc_opts *opts,
             void *stream);

/* pc_solve -- lowest nbands eigenpairs for each of nk Bloch vectors (Sections 3.2, 4.5, 5; Algorithm 4.1).
 *   kpts:   host [nk][3] Cartesian Bloch vectors in units 1/a (reduced internally: into [-pi, pi]^3 on the cube; by
 *           the reciprocal lattice G = 2 pi A^{-T} n, n = round(A^T k / 2 pi), on a general cell); a vector
 *           equivalent to 0 is treated as k = 0: its 3 constant kernel fields are projected out and the lowest
 *           nonzero eigenvalues are returned).
 *   nbands: eigenpairs per k-point, 1 <= nbands <= 21 (nbands + guard <= 21).
 *   tol:    column j converged when |Op x - lambda x| <= tol |lambda| |x|.
 *   evals:  host [nk][nbands] ascending omega^2 (units (1/a)^2).
 *   evecs:  device [nk][nbands][3][N][N][N] complex128, unit 2-norm, or NULL.
 *   iters:  host [nk] LOBPCG iterations (summed over gamma doublings), or NULL.
 *   resid:  host [nk][nbands] final relative residuals, or NULL.
 * All k-points are solved together (batched kernels). Returns PC_NOT_CONVERGED if some k-point hit maxiter and
 * PC_SPURIOUS if Algorithm 4.1 still saw a spurious eigenvalue after max_doublings (results are filled in both
 * cases). With PC_PREC_MIXED, a k-point whose FP64-accurate phase stops converging or reaches maxiter is solved
 * again by the FP64 solve, started from its current block (pc_get_fp64_finish tells which; its iteration count is
 * the sum of both). Synchronises the context stream before returning. */
int pc_solve(pc_ctx *ctx, int nk, const double *kpts, int nbands, double tol, double *evals, void *evecs,
             int *iters, double *resid);

/* pc_get_fp64_finish -- flags[b] = 1 for each k-point b of the last pc_solve / pc_solve_init on this context that
 * the mixed solve handed to the FP64 solve, 0 otherwise (all 0 after an FP64 solve).
 *   nk: the k-point count of that solve (PC_EINVAL otherwise); flags: host [nk]. No device work. */
int pc_get_fp64_finish(pc_ctx *ctx, int nk, int *flags);

/* pc_solve_init -- pc_solve from a caller-provided initial block: the first n0 columns of each k-point's starting
 * block are X0 (the learned warm start's prediction, or the eigenvectors of a neighbouring k-point), the remaining
 * columns are the counter-based random fields of pc_solve. At k = 0 the constant fields are projected out of X0 as
 * well. The paper's LOBPCG starts from a random block; this entry point has no counterpart there.
 *   X0: device complex64 [nk][n0][3][N][N][N]; 1 <= n0 <= nbands. Other arguments and results as pc_solve. */
int pc_solve_init(pc_ctx *ctx, int nk, const double *kpts, int nbands, double tol, const void *X0, int n0,
                  double *evals, void *evecs, int *iters, double *resid);

/* Release a context and its device memory (never caller memory). NULL is allowed. */
void pc_destroy(pc_ctx *ctx);

/* Thread-local description of the last error ("" if none). */
const char *pc_last_error(void);

/* ---------------- per-stage timing and launch counts (tracing) ---------------- */

/* Stages of a solve, in pc_stage_stat arrays. */
#define PC_STAGE_STENCIL 0   /* a1: Op X (fused stencil) */
#define PC_STAGE_PRECOND 1   /* a2: FFT preconditioner (5 kernels per call) */
#define PC_STAGE_GRAM 2      /* a3: Gram products S^H S, S^H AS */
#define PC_STAGE_RR 3        /* a4: Rayleigh-Ritz (small dense, one block per k-point) */
#define PC_STAGE_UPDATE 4    /* a5: block updates S C */
#define PC_STAGE_RESIDUAL 5  /* a5: residual and column norms */
#define PC_STAGE_RECOMPUTE 6 /* a6: Algorithm 4.1 norms */
#define PC_STAGE_OTHER 7     /* initial block, k = 0 projection */
#define PC_STAGE_DFLOAT 8    /* mixed solve, phase 2: double-float Op X, X-X Gram block and X update */
#define PC_NSTAGES 9

typedef struct {
    long calls;    /* stage invocations */
    long kernels;  /* kernel launches */
    double ms;     /* summed device time between CUDA events around each invocation (0 unless timing is on) */
    double flops;  /* algorithmic floating-point operations (real), summed */
    double bytes;  /* algorithmic global-memory bytes (each operand read once, each result written once) */
} pc_stage_stat;

/* Enable (1) or disable (0) event timing of every stage invocation of pc_solve on the context stream. Counts and
 * algorithmic work are always accumulated. */
int pc_set_timing(pc_ctx *ctx, int enable);
/* Copy the accumulated statistics (PC_NSTAGES entries) into out (host). */
int pc_get_stats(pc_ctx *ctx, pc_stage_stat *out);
/* Zero the accumulated statistics. */
int pc_reset_stats(pc_ctx *ctx);

/* ---------------- step-level entry points (the individual kernels of the solve) ---------------- */

/* a0: permittivity at the edge DoFs from a list of dielectric spheres (Section 4.4).
 *   spheres: host [nsph][5] = (cx, cy, cz, r, eps_in) in cell fractions; a point belongs to a sphere when its
 *            distance to a periodic image of the centre is <= r; later spheres take precedence.
 *   eps_bg:  permittivity outside all spheres.
 *   eps_out: host [3][N][N][N]. An edge midpoint within 1e-12 of a sphere surface takes the interface rule of
 *            Section 4.4: eps = (sum of eps at the 4 adjacent cell centres) / 4, so that M0 = 4 / sum.
 * Runs a device kernel; synchronous. */
int pc_eps_spheres(int N, int nsph, const double *spheres, double eps_bg, double *eps_out);

/* a0 on a general cell (Section 2's coordinate change x = A y; Section 4.4's rules).
 *   lattice: host double[9], a1, a2, a3 one after the other as in pc_setup; linearly independent (else PC_EINVAL).
 *   spheres: host [nsph][5] = (cx, cy, cz, r, eps_in), Cartesian (the units of the lattice vectors); a point x
 *            belongs to a sphere when its distance to the nearest image c + A n of the centre is <= r (images
 *            searched among the 27 translates around the reduced offset); later spheres take precedence.
 *   eps_out: host [3][N][N][N] at the points A y of the edge midpoints y of the unit cube; the interface rule of
 *            pc_eps_spheres applies with the cell centres mapped the same way.
 * Runs a device kernel; synchronous. */
int pc_eps_spheres_lattice(int N, const double *lattice, int nsph, const double *spheres, double eps_bg,
                           double *eps_out);

/* a0 for the structures of Section 6.3 on a general cell (lattice as in pc_setup; eps_out host [3][N][N][N] at the
 * Cartesian points A y of the edge midpoints y). Each runs a device kernel; synchronous.
 * pc_eps_gyroid: the single gyroid {g > threshold} with g = sin(2 pi x/l) cos(2 pi y/l) + sin(2 pi y/l) cos(2 pi z/l)
 *   + sin(2 pi z/l) cos(2 pi x/l) (Section 6.3: threshold 1.1, eps_in 16, in the BCC lattice of constant l); the
 *   strict inequality decides every point.
 * pc_eps_diamond: the FCC diamond: spheres of radius r l at (0,0,0) and (l/4)(1,1,1), and one spheroid per bond
 *   (l/4)(1,1,1), (l/4)(1,-1,-1), (l/4)(-1,1,-1), (l/4)(-1,-1,1) from the origin with foci at the bond's ends and
 *   minor axis of full length b l (Section 6.3: r = 0.12, b = 0.11, eps_in 13); closed sets, periodic images by the
 *   nearest-image search of pc_eps_spheres_lattice. */
int pc_eps_gyroid(int N, const double *lattice, double l, double threshold, double eps_in, double eps_bg,
                  double *eps_out);
int pc_eps_diamond(int N, const double *lattice, double l, double r, double b, double eps_in, double eps_bg,
                   double *eps_out);

/* a1: Y = Op X = A M0 A' X + gamma B'B X for nb k-points x m fields (eq. Ker_comp; stencils of Section 4.1.2,
 * of the context's order: Table 1's 2k-th order schemes).
 *   kpts: host [nb][3] (used as given, no zone reduction); gammas: host [nb].
 *   X, Y: device blocks, dtype PC_C128, PC_C64 or PC_C128_DF (complex128 data, double-float arithmetic; order 1
 *         only), batch stride m*3N^3 elements. X and Y must not overlap. Orders above 1 use a scratch block of
 *         4 m N^3 entries per k-point owned by the context. */
int pc_apply_op(pc_ctx *ctx, int nb, const double *kpts, const double *gammas, int m, int dtype, const void *X,
                void *Y);

/* a1h: E = A' X (faces -> edges, [m][3][N^3]) and C = B X (faces -> cells, [m][N^3]) per k-point (Section 4.3,
 * eq. derived_uniform_grid). dtype PC_C128 only. Batch strides m*3N^3 (E) and m*N^3 (C). Either output may be NULL. */
int pc_apply_half(pc_ctx *ctx, int nb, const double *kpts, int m, const void *X, void *E, void *C);

/* a6: the norms of Algorithm 4.1 for each field x of the blocks (PC_C128):
 *   out (device double [nb][m][3]) = (|M0^{1/2} A' x|^2, |B x|^2, |x|^2).
 * lambda_re = out[0]/out[2]; the symmetric Rayleigh quotient is (out[0] + gamma out[1]) / out[2]. */
int pc_recompute_norms(pc_ctx *ctx, int nb, const double *kpts, int m, const void *X, double *out);

/* Table 1: the weights of the 2k-th order staggered difference (c_s) and midpoint average (d_s), s = 1..4 (zero
 * past k), for order = k in 1..4 (c, d: host double[4]). Host only. PC_EINVAL for another order. */
int pc_stencil_coefficients(int order, double *c, double *d);

/* a2: W = P^{-1} R with P = A A' + gamma B'B (or the vector Laplacian, per opts.precond): forward 3D FFT, the exact
 * inverse of the 3x3 symbol sigma I + (gamma-1) conj(d) d^T per mode, inverse 3D FFT (Algorithm 5.1,
 * eq. penalised_marix). At k = 0 the singular mode 0 is mapped to 0. R and W may be the same buffer (in place). */
int pc_apply_precond(pc_ctx *ctx, int nb, const double *kpts, const double *gammas, int m, int dtype,
                     const void *R, void *W);

/* a3: G_b = A_b^H B_b for tall-skinny blocks (L rows; p and q columns, column stride L; batch strides sa, sb in
 * elements). G: device complex128 [nb][p][q] row-major. p, q <= 64. dtype applies to A and B. PC_C128: FP64
 * products and sums. PC_C64: FP32 products and partial sums over chunks of the rows, chunks added in FP64; where L
 * is a multiple of 16 and the panels are 16-byte aligned this runs on the tensor cores (TF32 operands split into
 * hi + lo, accumulators drained every 64 rows), otherwise on the CUDA cores. */
int pc_gram(int nb, long L, int p, int q, int dtype, const void *A, long sa, const void *B, long sb, void *G,
            void *stream);

/* a3: the Rayleigh-Ritz pencil of one panel: G_b = S_b^H S_b and H_b = S_b^H AS_b, with S_b and AS_b of p columns
 * (length L, column stride L, the same batch stride ss for both). Op is Hermitian, so both outputs are Hermitian:
 * only the upper triangle is accumulated (FP64) and the lower triangle is its conjugate mirror. G, H: device
 * complex128 [nb][p][p]. p <= 64; dtype applies to S and AS, with the accumulation of pc_gram for that dtype. */
int pc_gram_pair(int nb, long L, int p, int dtype, const void *S, long ss, const void *AS, void *G, void *H,
                 void *stream);

/* a3 with the mixed solve's coupling block: G_b = S_b^H S_b, H_b = S_b^H AS_b (as pc_gram_pair) and
 * RQ_b = R_b^H S_b (q x p, complex128 [nb][q][p]) from one pass over S, AS and R (complex64 only; R_b of q columns,
 * batch stride sr). The coupling X^H Op Q = Theta X^H Q + R^H Q of Section 5.1's LOBPCG takes R^H Q from RQ.
 * p, q <= 64; on the tensor cores when 2 round8(p) + round8(q) <= 128 (rounded to 16), else as pc_gram_pair plus
 * pc_gram. Synchronous. */
int pc_gram_pair_coupled(int nb, long L, int p, int q, const void *S, long ss, const void *AS, const void *R, long sr,
                         void *G, void *H, void *RQ, void *stream);

/* pc_gram_pair_noalloc -- the same products as pc_gram_pair, for callers that cannot allocate device memory:
 * code that runs under a fixed device-memory budget, inside an application whose own allocator must own every
 * allocation, or in latency-critical loops where cudaMalloc/cudaFree would synchronise the device. It calls no
 * cudaMalloc, cudaFree or other allocating routine; its partial sums live in a 4 MiB array that is part of the
 * library image, so every GPU that loads the library holds those 4 MiB until the process exits.
 * This entry point has no counterpart in the paper; it is an interface convenience.
 *   Limit: 2 * 16 * nb * p * p <= 4 MiB, i.e. nb * p * p <= 131072 (for example 32 k-points of 64 columns);
 *   larger requests return PC_EINVAL with a message. Arguments and layout are those of pc_gram_pair. Results agree
 *   with pc_gram_pair within rounding, but not bit for bit: complex64 panels are always summed on the CUDA cores
 *   (FP32 products and partial sums over row chunks, chunks added in FP64), never on the tensor-core path that
 *   pc_gram_pair takes for them. The call is asynchronous: it returns once the work is enqueued on `stream`
 *   (pc_gram_pair waits for its stream), so G and H are valid only after the caller synchronises with `stream`.
 *   The first call on each device looks up the array's device address (cudaGetSymbolAddress) with that device
 *   current; make that first call before any stream capture. Every call reuses the same array and only reads
 *   entries it has written itself, so no state carries over between calls, but calls whose work overlaps on the
 *   GPU (other streams, other host threads) race on the array and must be serialised by the caller. */
int pc_gram_pair_noalloc(int nb, long L, int p, int dtype, const void *S, long ss, const void *AS, void *G, void *H,
                         void *stream);

/* a5: Y_b = S_b C_b: S_b has p columns of length L (batch stride ss), C_b device complex128 [p][q] row-major
 * (batch stride p*q), Y_b has q columns (batch stride sy). p <= 64, q <= 64. dtype applies to S and Y. */
int pc_block_update(int nb, long L, int p, int q, int dtype, const void *S, long ss, const void *C, void *Y,
                    long sy, void *stream);

/* a4: batched Hermitian eigensolver (cyclic Jacobi, FP64) of device complex128 A [nb][n][n] (row-major, only the
 * Hermitian part is used); w: device double [nb][n] ascending; V: device complex128 [nb][n][n], column j is the
 * eigenvector of w[j]. n <= 64. */
int pc_eigh_batched(int nb, int n, const void *A, double *w, void *V, void *stream);

/* a4: Rayleigh-Ritz on span(S) for nb pencils (H, G) = (S^H Op S, S^H S), each n x n (device complex128, batch
 * stride n*n): scale to unit diagonal, orthonormalise through the eigenvectors of G (dropping directions with
 * eigenvalue < drop * max), solve the projected problem and return the lowest m Ritz values theta (device double
 * [nb][m]) and coefficients coef (device complex128 [nb][n][m], so that S coef are the Ritz vectors; unit-norm
 * and mutually orthogonal). rank (device int [nb], or NULL) receives the retained dimension. */
int pc_rayleigh_ritz(int nb, int n, int m, const void *G, const void *H, double drop, double *theta, void *coef,
                     int *rank, void *stream);

/* a5: R = AX - X diag(theta) and column norms norms (device double [nb][m][2]) = (|r_j|, |x_j|). Blocks of m
 * columns, batch stride m*L, dtype PC_C128. theta device double [nb][m]. */
int pc_residual(int nb, long L, int m, const void *X, const void *AX, const double *theta, void *R,
                double *norms, void *stream);

/* Initial block: field j of k-point b is the counter-based complex normal stream (seed, (kidx0+b)*4096 + j)
 * (splitmix64 output function + Box-Muller; see the oracle's rng module for the definition). Device PC_C128. */
int pc_init_block(int nb, long L, int m, uint64_t seed, int kidx0, void *X, void *stream);

/* ---------------- learned warm start (no counterpart in the paper; its LOBPCG starts from a random block) -------
 * A 3D convolutional network over M0 = 1/eps, conditioned on k, predicts an initial block X0 of nb face fields and
 * guesses y of log lambda for nb bands: conv 3 -> PC_WS_C1 and PC_WS_C1 -> PC_WS_C2 channels (3x3x3, stride 2,
 * circular padding, bias, ReLU), FiLM from phi(k) = (sin k, cos k), a 1x1x1 head to 6 nb channels at (N/4)^3,
 * periodic linear upsampling x4 per axis; value head y = Wv [mean z; phi] + bv. Trained by the subspace loss
 * nb - tr(G^-1 B B^H), G = X^H X, B = X^H V, against eigenvectors V of converged solves, plus w_val (y - log lambda)^2.
 * All network arithmetic is FP32; the Grams accumulate in FP64.
 * Parameters: one flat device float array of pc_ws_param_count(nb) entries in the order W1 (C1,3,3,3,3), b1,
 * W2 (C2,C1,3,3,3), b2, Fa (C2,6), fa, Fc (C2,6), fc, Wh (6 nb, C2), bh, Wv (nb, C2 + 6), bv, each row-major.
 * Sizes: N a power of two in [16, 256]; 1 <= nb <= 16; 1 <= S <= 65535 samples per call. */
#define PC_WS_C1 8
#define PC_WS_C2 16

/* Number of floats in the parameter array for nb bands (-1 if nb is out of range). Host only. */
long pc_ws_param_count(int nb);

/* Bytes of the device workspace that pc_ws_forward and pc_ws_backward share for S samples (0 if out of range). */
size_t pc_ws_work_bytes(int N, int nb, int S);

/* Forward pass for S samples.
 *   params: device float [pc_ws_param_count(nb)].
 *   m0:     device float [nstruct][3][N][N][N], M0 = 1/eps at the edge DoFs of each structure.
 *   sidx:   device int [S], the structure of each sample, each in [0, nstruct) (checked on the host: PC_EINVAL).
 *   kpts:   host double [S][3], the Bloch vector of each sample.
 *   X:      device complex64 [S][nb][3][N][N][N] (out): the predicted block of each sample.
 *   y:      device float [S][nb] (out): the guesses of log lambda.
 *   work:   device buffer of pc_ws_work_bytes(N, nb, S) bytes; keeps the activations for pc_ws_backward.
 * Synchronous on stream. */
int pc_ws_forward(int N, int nb, int S, const float *params, const float *m0, int nstruct, const int *sidx,
                  const double *kpts, void *X, float *y, void *work, void *stream);

/* Loss and gradient for the S samples of the preceding pc_ws_forward call with the same work buffer and inputs.
 *   V:     device complex64 [S][nb][3][N][N][N], orthonormal eigenvectors of each sample's converged solve.
 *   lam:   device double [S][nb], the eigenvalues (> 0).
 *   grad:  device float [pc_ws_param_count(nb)] (out): the gradient of the mean loss over the S samples.
 *   loss:  device double [S] (out): each sample's loss (NaN where X^H X was not positive definite; that sample
 *          then adds no gradient).
 * Enqueued on stream; returns before completion. */
int pc_ws_backward(int N, int nb, int S, const float *params, const float *m0, int nstruct, const int *sidx,
                   const void *X, const float *y, const void *V, const double *lam, float w_val, float *grad,
                   double *loss, void *work, void *stream);

/* One Adam step (Kingma and Ba) on P parameters in place: m, v device float [P] moments (zero before step t = 1),
 * t the 1-based step count for the bias corrections. Enqueued on stream. */
int pc_ws_adam(long P, float *params, const float *grad, float *m, float *v, int t, float lr, float b1, float b2,
               float eps, void *stream);

#ifdef __cplusplus
}
#endif
#endif
