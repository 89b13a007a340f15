// Internal helpers shared by the libpc translation units: complex arithmetic on interleaved pairs, error state,
// per-k-point parameters and the context layout.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "pc.h"

namespace pc {

// ---------------------------------------------------------------- complex on (x = re, y = im) pairs
template <typename T> struct cplx_of;
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<float> { using type = float2; };
template <typename T> using cplx = typename cplx_of<T>::type;

template <typename C> __host__ __device__ __forceinline__ C cmake(decltype(C{}.x) re, decltype(C{}.x) im) {
  C r;
  r.x = re;
  r.y = im;
  return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  return cmake<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) {
  return cmake<C>(a.x * s, a.y * s);
}

// ---------------------------------------------------------------- per-k-point parameters
struct KParam {
  double k[3];   // Bloch vector (units 1/a)
  double gamma;  // penalty of eq. pnt_number
  float khf[3];  // k_i / 2 and gamma rounded to FP32, so that complex64 kernels do no FP64 arithmetic
  float gammaf;
  float khl[3];  // remainders: (khf, khl) and (gammaf, gammal) are the double-float values of k_i / 2 and gamma
  float gammal;
  float pfacf;   // (gamma - 1) / gamma rounded to FP32 (the complex64 preconditioner's projection factor)
};

// internal dtype of the mixed solve's FP64-accurate block: complex double-float pairs, one float4 per element
// (re.hi, re.lo, im.hi, im.lo); never passed through the C ABI
constexpr int PC_DFS = 3;

// ---------------------------------------------------------------- error state
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define PC_CK(call)                                                   \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return pc::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)
#define PC_CK_LAUNCH() PC_CK(cudaGetLastError())
#define PC_REQUIRE(cond, ...)       \
  do {                              \
    if (!(cond)) {                  \
      pc::set_error(__VA_ARGS__);   \
      return PC_EINVAL;             \
    }                               \
  } while (0)

inline int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}
inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Streaming multiprocessors of the current device (queried once per device): grids and chunk counts are sized in
// multiples of it. Falls back to 1 if the query fails, so that sizes stay valid.
inline int sm_count() {
  static int count[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (count[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    count[dev] = n;
  }
  return count[dev];
}

// ---------------------------------------------------------------- device buffer that frees itself
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // grows (never shrinks) to at least nbytes; returns cudaSuccess or the allocation error
  cudaError_t reserve(size_t nbytes) {
    if (nbytes <= bytes) return cudaSuccess;
    release();
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = nbytes;
    return cudaSuccess;
  }
  template <typename T> T *as() const { return static_cast<T *>(p); }
};

}  // namespace pc

// ---------------------------------------------------------------- the context
struct pc_ctx {
  int N = 0, logN = 0;
  long n = 0;  // N^3
  pc_opts opts{};
  cudaStream_t stream = nullptr;
  // general lattice (Section 2's coordinate change x = A y, Section 4.2.2): lat is set when A is not the identity;
  // binv = A^{-1} row-major (binv[3 * i + j] = b_ij), amat = A row-major (amat[3 * i + j] = a_j component i)
  bool lat = false;
  // caller-provided initial block of pc_solve_init: device complex64 [nk][x0n][3][N][N][N], or null; complex128
  // when x0_c128 is set (the mixed solve's FP64 finish hands its double-float blocks to the FP64 solve that way)
  const void *x0 = nullptr;
  int x0n = 0;
  bool x0_c128 = false;
  // per k-point of the last pc_solve: 1 where the mixed solve handed the k-point to the FP64 solve (FP64 finish)
  std::vector<int> fp64_finish;
  pc::DevBuf finbuf;  // FP64 finish: the handed-over blocks (complex128) and the finished eigenvectors
  // index of the batch's first k-point within the caller's list: a chunked pc_solve passes each chunk's offset, so
  // that every k-point draws the initial columns of its own index (the same block as in an unchunked solve)
  int kidx0 = 0;
  double binv[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double amat[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  pc::DevBuf m0d, m0f;      // M0 diagonal, double and float copies, [3][N^3]
  pc::DevBuf m0p;           // M0 diagonal as double-float pairs (hi, lo) float2 [3][N^3]
  pc::DevBuf kscratch;      // two-pass stencils: e = M0 A' v (3 fields) and c = B v (1 field) per column
  pc::DevBuf kscratch_x[3]; // the same for k-point groups 1.. of the mixed solve (their own streams, concurrent)
  pc::DevBuf twd, twf;      // FFT twiddles exp(-2 pi i t / N), t < N/2
  pc::DevBuf kparam;        // KParam [nb]
  pc::DevBuf symd;          // per-k axis symbols d_i(m) complex128 [nb][3][N]; general lattice: [nb][3][3][N]
  pc::DevBuf scratch;       // general scratch (partial sums)
  int kcap = 0;             // capacity (k-points) of kparam / symd
  // solver buffers
  pc::DevBuf S[2], AS[2], Gm, Hm, coef, theta, norms, rnorm, rank, flag;
  // mixed-precision solve: FP64 block X, complex64 residual copy, coupling R^H S, FP64 X^H X, phases, masks
  pc::DevBuf X64[2], R32, RQ, GX, phase, mask;
  // mixed solve with several k-point groups: the streams of groups 1.. (group 0 runs on `stream`), and pinned host
  // copies of theta, column norms and Algorithm 4.1 norms (so that a group's device-to-host copies do not block the
  // host)
  static constexpr int kMaxGroups = 4;
  cudaStream_t xstream[kMaxGroups - 1] = {};
  // per group: a stream of the highest priority for its Rayleigh-Ritz launches (few blocks, latency-bound), so that
  // their blocks take SMs ahead of the pending blocks of other groups' large grids
  cudaStream_t rrstream[kMaxGroups] = {};
  double *pinned = nullptr;
  size_t pinned_count = 0;
  // tracing: per-stage statistics and event pairs awaiting harvest
  bool timing = false;
  pc_stage_stat stats[PC_NSTAGES] = {};
  struct Pending {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  ~pc_ctx() {
    for (cudaStream_t s : xstream)
      if (s) cudaStreamDestroy(s);
    for (cudaStream_t s : rrstream)
      if (s) cudaStreamDestroy(s);
    if (pinned) cudaFreeHost(pinned);
    for (auto &p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : event_pool) cudaEventDestroy(e);
  }
};

namespace pc {
// The two-pass stencils' scratch for the stream the context currently issues on: the mixed solve's k-point groups
// run concurrently on their own streams, each with its own buffer; every other caller uses ctx->kscratch.
static_assert(sizeof(pc_ctx::kscratch_x) / sizeof(DevBuf) == pc_ctx::kMaxGroups - 1, "one scratch per extra group");
inline DevBuf &kscratch_for(pc_ctx *ctx) {
  for (int i = 0; i < pc_ctx::kMaxGroups - 1; ++i)
    if (ctx->xstream[i] && ctx->stream == ctx->xstream[i]) return ctx->kscratch_x[i];
  return ctx->kscratch;
}
// Runs one stage invocation: counts it, adds its algorithmic work, and brackets it with events when timing is on.
template <typename F> int run_stage(pc_ctx *ctx, int stage, int kernels, double flops, double bytes, F &&launch);
// Accumulates the elapsed times of finished event pairs; pairs still in flight stay pending.
int harvest_timing(pc_ctx *ctx);
// A (row-major) and b = A^{-1} (row-major) from the lattice vectors a_1, a_2, a_3 stored one after the other
// (lattice[3 n + c] = component c of a_{n+1}); nonzero when the vectors are numerically dependent
int invert_lattice(const double *lattice, double *amat, double *binv);
// uploads kparams (and symbol tables) for nb k-points into the context; returns 0 or an error code
int upload_kpoints(pc_ctx *ctx, int nb, const double *kpts, const double *gammas);
// kernels launched by the solver (all on ctx->stream)
int launch_apply_op(pc_ctx *ctx, int nb, int m, int dtype, const void *X, long sx, void *Y, long sy,
                    const int *act);
int launch_precond(pc_ctx *ctx, int nb, int m, int dtype, const void *R, long sr, void *W, long sw,
                   const int *act);
// complex64 preconditioner in three natural-order passes (fft_c64.cu); PC_EUNSUPPORTED for sizes it does not take
int launch_precond_c64(pc_ctx *ctx, int nb, int m, const void *R, long sr, void *W, long sw, const int *act);
// nb_alloc: k-points in the panel arrays (the act list indexes them); <= 0 means nb.
// sg: batch stride of the output matrices in elements; <= 0 means packed (p q, or p p for the pair).
int launch_gram(int nb, long L, int p, int q, int dtype, const void *A, long sa, const void *B, long sb, void *G,
                void *scratch, size_t scratch_bytes, cudaStream_t st, const int *act, int nb_alloc = -1,
                long sg = 0);
size_t gram_scratch_bytes(int nb, long L, int p, int q);
int launch_gram_pair(int nb, long L, int p, int dtype, const void *S, const void *AS, long ss, void *G, void *H,
                     void *scratch, size_t scratch_bytes, cudaStream_t st, const int *act, int nb_alloc = -1,
                     long sg = 0);
size_t gram_pair_scratch_bytes(int nb, long L, int p);
// reductions of per-chunk partial sums ([nb][nchunk][p][q] double2; the pair: G block then H block, upper triangles)
void launch_gram_pair_reduce(int nb, int nchunk, int p, const double2 *part, const int *act, void *G, void *H,
                             cudaStream_t st, long sg = 0);
void launch_gram_reduce(int nb, int nchunk, int p, int q, const double2 *part, const int *act, void *G,
                        cudaStream_t st, long sg = 0);
// complex64 Gram products on the tensor cores (gram_tc.cu); PC_EUNSUPPORTED when the shape does not fit
int launch_gram_pair_tc(int nb, long L, int p, const void *S, const void *AS, long ss, void *G, void *H,
                        void *scratch, size_t scratch_bytes, cudaStream_t st, const int *act, int nb_alloc, long sg);
int launch_gram_pair_coupled_tc(int nb, long L, int p, int q2, const void *S, const void *AS, long ss, const void *R,
                                long sr, void *G, void *H, void *RQ, void *scratch, size_t scratch_bytes,
                                cudaStream_t st, const int *act, int nb_alloc, long sg, long srq);
// G = S^H S, H = S^H AS (p columns) and RQ = R^H S (q2 x p) for nb k-points; one tensor-core pass for complex64
// where the shape allows, else launch_gram_pair and launch_gram
int launch_gram_pair_coupled(int nb, long L, int p, int q2, int dtype, const void *S, const void *AS, long ss,
                             const void *R, long sr, void *G, void *H, void *RQ, void *scratch, size_t scratch_bytes,
                             cudaStream_t st, const int *act, int nb_alloc = -1, long sg = 0, long srq = 0);
size_t gram_pair_coupled_scratch_bytes(int nb, long L, int p, int q2);
int launch_gram_tc(int nb, long L, int p, int q, const void *A, long sa, const void *B, long sb, void *G,
                   void *scratch, size_t scratch_bytes, cudaStream_t st, const int *act, int nb_alloc, long sg);
// chunks per k-point that the tensor-core Gram takes at least for panels of L rows (its partial sums need that many)
int tc_min_chunks(long L);
// reads and clears the time-out flag of the tensor-core Gram kernel (call after a synchronisation)
int gram_tc_check();
// Y = S C (+ Z, a complex64 addend, if Z is not null); arithmetic in the precision of dtype
int launch_block_update(int nb, long L, int p, int q, int dtype, const void *S, long ss, const void *C, long sc,
                        void *Y, long sy, cudaStream_t st, const int *act, const void *Z = nullptr, long sz = 0);
// sg, sc: batch strides of G/H and of coef in elements; <= 0 means packed (n n, n m)
int launch_rr(int nb, int n, int m, const void *G, const void *H, double drop, double *theta, void *coef,
              int *rank, cudaStream_t st, const int *act, long sg = 0, long sc = 0);
// algorithmic FP64 flops of one Rayleigh-Ritz pencil of n columns, m wanted pairs (Cholesky, the two substitutions,
// Householder tridiagonalisation, back-transformation; bisection and inverse iteration are of lower order)
double rr_flops(int n, int m);
int launch_residual(int nb, long L, int m, const void *X, long sx, const void *AX, long sax, const double *theta,
                    void *R, long sr, double *norms, void *scratch, size_t scratch_bytes, cudaStream_t st,
                    const int *act);
size_t residual_scratch_bytes(int nb, long L, int m);
// X: dtype PC_C128 (complex128) or PC_DFS (double-float pairs)
int launch_recompute(pc_ctx *ctx, int nb, int m, const void *X, long sx, double *out, const int *act, void *scratch,
                     size_t scratch_bytes, int dtype = PC_C128);
size_t recompute_scratch_bytes(long n, int nb, int m);
int launch_deflate(int nb, long n, int m, void *X, long sx, const int *flags, void *scratch, cudaStream_t st,
                   const int *act, int dtype = PC_C128);
size_t deflate_scratch_bytes(int nb, int m);
int launch_residual_mixed(int nb, long L, int m, int dtype_x, const void *X, long sx, const void *AX, long sax,
                          const double *theta, void *R1, long sr1, void *R2, long sr2, void *X32, long sx32,
                          void *AX32, long sax32, double *norms, void *scratch, size_t scratch_bytes,
                          cudaStream_t st, const int *act);
int launch_rr_patch(int nb, int n, int m, void *G, void *H, const void *RS, const double *theta, const void *GX,
                    const int *phase, cudaStream_t st, const int *act, long sg = 0, long srs = 0);
int launch_widen(int nb, long L, int m, const void *X, long sx, void *Y, long sy, cudaStream_t st, const int *act);
// Y (complex128) = X (double-float pairs, PC_DFS): m columns of length L per k-point
int launch_pairs_to_c128(int nb, long L, int m, const void *X, long sx, void *Y, long sy, cudaStream_t st,
                         const int *act);
// stencils of order k = 2..4 (stencil_k.cu): Table 1 coefficients (c_s, d_s, s <= 4, zero past k), Y = Op X in two
// passes (complex128 or complex64), the half-apply (A' x, B x; complex128) and the Algorithm 4.1 partial sums
void stencil_coefficients(int k, double *c, double *d);
int launch_apply_op_k(pc_ctx *ctx, int nb, int m, int dtype, const void *X, long sx, void *Y, long sy,
                      const int *act);
int launch_half_k(pc_ctx *ctx, int nb, int m, const void *X, void *E, void *Cc);
int launch_recompute_k_partial(pc_ctx *ctx, int nb, int m, const void *X, long sx, const int *act, int nchunk,
                               long chunk, double *part, int dtype);
// The two-pass kernels above also serve a general lattice (ctx->lat) at every order 1..4: D_hat_a = sum_j b_ja K_j
// + i L_a replaces D_a (Section 4.2.2).
// double-float (FP32-pair) versions of the FP64-accurate kernels of the mixed solve (mixed_df.cu). launch_apply_op_df
// takes complex128 blocks; the others take and write blocks of double-float pairs (PC_DFS).
int launch_apply_op_df(pc_ctx *ctx, int nb, int m, const void *X, long sx, void *Y, long sy, const int *act);
// the same stencil with the residual epilogue of the mixed solve's phase 2 instead of writing AX: complex64
// r = AX - X Theta into R1 and R2, complex64 copies of X and AX, column norms (|r|, |x|) into norms [nb][m][2]
int launch_op_df_resid(pc_ctx *ctx, int nb, int m, const void *X, long sx, const double *theta, void *R1, long sr1,
                       void *R2, long sr2, void *X32, long sx32, void *AX32, long sax32, double *norms, void *scratch,
                       size_t scratch_bytes, const int *act);
size_t op_df_resid_scratch_bytes(pc_ctx *ctx, int nb, int m);
void launch_residual_reduce(int nb, int nchunk, int m, const double *part, const int *act, double *norms,
                            cudaStream_t st);
int launch_update_df(int nb, long L, int p, int q, const void *X, long sx, const void *C, long sc, void *Y, long sy,
                     const void *Z, long sz, cudaStream_t st, const int *act);
// G = X^H X of a block of double-float pairs (p <= 32 columns) in double-float arithmetic, G complex128
int launch_gram_df(int nb, long L, int p, const void *X, long sx, void *G, void *scratch, size_t scratch_bytes,
                   cudaStream_t st, const int *act);
size_t gram_df_scratch_bytes(int nb, long L, int p);
// the mixed-precision LOBPCG driver (solver_mixed.cu); k-points already reduced, gammas per k-point
// k-points whose phase 2 stalled or reached maxiter are not finished: their indices and the buffer (0 or 1 of
// ctx->X64) that holds their double-float block are appended to `handover`, for the FP64 finish of pc_solve
int solve_mixed(pc_ctx *ctx, int nb, const double *kr, std::vector<double> &gam, const std::vector<int> &zero,
                int nbands, int m, double tol, double *evals, void *evecs, int *iters, double *resid,
                std::vector<std::pair<int, int>> *handover);
// counter-based initial columns; with mask (int [nb][m]) only the flagged columns of the act k-points are written
// X: dtype PC_C128, PC_DFS (the same FP64 values stored as double-float pairs) or PC_C64 (the same uniforms, the
// normal deviates formed in FP32)
// the caller's initial block (ctx->x0, complex64 or, with ctx->x0_c128, complex128) into the first ctx->x0n
// columns of the panels of k-points
// b0 .. b0 + nbk - 1 at X + b * sx (dtype PC_C128 or PC_C64 panels; sx in elements)
int launch_copy_x0(const pc_ctx *ctx, int b0, int nbk, int dtype, void *X, long sx, cudaStream_t st);
int launch_init_block(int nb, long L, int m, uint64_t seed, int kidx0, void *X, long sx, cudaStream_t st,
                      const int *mask = nullptr, const int *act = nullptr, int dtype = PC_C128);
// Algorithm 4.1 restart: flags (host, [nb][m]) the columns of the redo k-points to replace before the re-solve
void spurious_mask(const std::vector<int> &redo, int m, int nbands, double tol, const std::vector<double> &theta,
                   const std::vector<double> &rn, std::vector<int> &mask);
}  // namespace pc

namespace pc {
cudaError_t get_event(pc_ctx *ctx, cudaEvent_t *e);

template <typename F> int run_stage(pc_ctx *ctx, int stage, int kernels, double flops, double bytes, F &&launch) {
  pc_stage_stat &st = ctx->stats[stage];
  st.calls += 1;
  st.kernels += kernels;
  st.flops += flops;
  st.bytes += bytes;
  if (!ctx->timing) return launch();
  cudaEvent_t a, b;
  PC_CK(get_event(ctx, &a));
  PC_CK(get_event(ctx, &b));
  PC_CK(cudaEventRecord(a, ctx->stream));
  int rc = launch();
  PC_CK(cudaEventRecord(b, ctx->stream));
  ctx->pending.push_back({stage, a, b});
  return rc;
}
}  // namespace pc
