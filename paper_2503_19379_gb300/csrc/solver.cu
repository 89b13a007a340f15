// Context management and the batched LOBPCG driver of pc_solve (Sections 3.2, 4.5 and 5; Algorithm 4.1).
//
// Per k-point the state is two ping-pong panels S = [X | W | P] and AS = [AX | AW | AP] of 3m columns each
// (m = nbands + guard, L = 3N^3 rows). One iteration, for all unconverged k-points at once:
//   R = AX - X Theta (into the W slot) and column norms       -> host convergence test
//   W = P^{-1} R (FFT preconditioner), AW = Op W
//   G = S^H S, H = S^H AS                                       (Gram products, 2m or 3m columns)
//   Rayleigh-Ritz on (H, G) -> Theta, coef                      (one thread block per k-point)
//   X' = S coef, P' = [W P] coef_{W,P}                          (into the other panel)
//   AX' = Op X', AP' = Op P'                                    (recomputed by the stencil: no drift)
// When a k-point converges, Algorithm 4.1 recomputes lambda_re = |M0^{1/2} A' x|^2 / |x|^2; if some value differs
// from its Ritz value (|lambda - lambda_re| > 10 tol lambda), gamma is doubled and the k-point keeps iterating
// from its current block (AX and AP recomputed with the new gamma).
// At k = 0 the constant fields (the kernel, Remark in Section 5.1) are projected out of X, W and P.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "pc_internal.cuh"

namespace pc {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  return e == cudaErrorMemoryAllocation ? PC_ENOMEM : PC_ECUDA;
}

// symbol of D_i on mode m for the 2k-th order stencil (Section 5.2, the diagonalisation of the difference and average
// matrices by the FFT): d_i(m) = i e^{i th/2} (S_i(m) + k_i Z_i(m)), th = 2 pi m / N, with
// S_i(m) = (2/h) sum_s c_s sin((s - 1/2) th) and Z_i(m) = 2 sum_s d_s cos((s - 1/2) th); for k = 1 (c_1 = 1,
// d_1 = 1/2) this is i e^{i th/2} ((2/h) sin(th/2) + k_i cos(th/2))
static void axis_symbols(int N, int order, double k_i, double2 *out) {
  const double h = 1.0 / N;
  double c[4], d[4];
  stencil_coefficients(order, c, d);
  for (int mm = 0; mm < N; ++mm) {
    const double th = 2.0 * M_PI * mm / N;
    double S = 0.0, Z = 0.0;
    for (int q = 1; q <= order; ++q) {
      S += c[q - 1] * std::sin((q - 0.5) * th);
      Z += d[q - 1] * std::cos((q - 0.5) * th);
    }
    const double mag = (2.0 / h) * S + k_i * (2.0 * Z);
    // i e^{i th/2} = -sin(th/2) + i cos(th/2)
    out[mm].x = -std::sin(0.5 * th) * mag;
    out[mm].y = std::cos(0.5 * th) * mag;
  }
}

// General lattice (Section 4.2.2): D_hat_i = sum_j b_ji K_j + i L_i has the symbol
// d_i = sum_j i e^{i th_j/2} (b_ji S(m_j) + [j = i] k_i Z(m_j)), a sum of one table per axis j. This writes the table
// of axis j for component i: weights wS = b_ji and wZ = k_i (j = i) or 0.
static void lattice_part_symbols(int N, int order, double wS, double wZ, double2 *out) {
  const double h = 1.0 / N;
  double c[4], d[4];
  stencil_coefficients(order, c, d);
  for (int mm = 0; mm < N; ++mm) {
    const double th = 2.0 * M_PI * mm / N;
    double S = 0.0, Z = 0.0;
    for (int q = 1; q <= order; ++q) {
      S += c[q - 1] * std::sin((q - 0.5) * th);
      Z += d[q - 1] * std::cos((q - 0.5) * th);
    }
    const double mag = wS * ((2.0 / h) * S) + wZ * (2.0 * Z);
    out[mm].x = -std::sin(0.5 * th) * mag;
    out[mm].y = std::cos(0.5 * th) * mag;
  }
}

// amat[3 i + j] = component i of a_{j+1}; b = A^{-1} by the adjugate
int invert_lattice(const double *lattice, double *amat, double *binv) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) amat[3 * i + j] = lattice[3 * j + i];
  const double *a = amat;
  const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  double scale = 0.0;
  for (int i = 0; i < 9; ++i) scale = std::max(scale, std::fabs(a[i]));
  if (!(std::fabs(det) > 1e-12 * scale * scale * scale)) return 1;
  // adjugate / det
  binv[0] = c00 / det;
  binv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  binv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  binv[3] = c01 / det;
  binv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  binv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  binv[6] = c02 / det;
  binv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  binv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
  return 0;
}

void spurious_mask(const std::vector<int> &redo, int m, int nbands, double tol, const std::vector<double> &theta,
                   const std::vector<double> &rn, std::vector<int> &mask) {
  std::fill(mask.begin(), mask.end(), 0);
  for (int b : redo)
    for (int j = 0; j < m; ++j) {
      const double *o = &rn[((size_t)b * m + j) * 3];
      const double lre = o[0] / o[2], lam = theta[(size_t)b * m + j];
      // first nbands: the equality test of Algorithm 4.1; guard columns (not converged): compensation-dominated
      const bool bad = j < nbands ? std::fabs(lam - lre) > 10.0 * tol * std::fabs(lam) : lre < 0.5 * lam;
      mask[(size_t)b * m + j] = bad ? 1 : 0;
    }
}

int upload_kpoints(pc_ctx *ctx, int nb, const double *kpts, const double *gammas) {
  if (nb <= 0) return PC_OK;
  const int tabs = ctx->lat ? 9 : 3;  // symbol tables per k-point: d_i by axis, or the parts (i, j) of d_i
  if (nb > ctx->kcap) {
    PC_CK(ctx->kparam.reserve(sizeof(KParam) * nb));
    PC_CK(ctx->symd.reserve(sizeof(double2) * tabs * (size_t)ctx->N * nb));
    ctx->kcap = nb;
  }
  std::vector<KParam> kp(nb);
  std::vector<double2> sym((size_t)tabs * ctx->N * nb);
  for (int b = 0; b < nb; ++b) {
    for (int d = 0; d < 3; ++d) {
      kp[b].k[d] = kpts[3 * b + d];
      kp[b].khf[d] = (float)(0.5 * kpts[3 * b + d]);
      kp[b].khl[d] = (float)(0.5 * kpts[3 * b + d] - (double)kp[b].khf[d]);
    }
    kp[b].gamma = gammas[b];
    kp[b].gammaf = (float)gammas[b];
    kp[b].gammal = (float)(gammas[b] - (double)kp[b].gammaf);
    kp[b].pfacf = (float)((gammas[b] - 1.0) / gammas[b]);
    if (!ctx->lat) {
      for (int d = 0; d < 3; ++d)
        axis_symbols(ctx->N, ctx->opts.order, kpts[3 * b + d], &sym[((size_t)b * 3 + d) * ctx->N]);
    } else {
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          lattice_part_symbols(ctx->N, ctx->opts.order, ctx->binv[3 * j + i], j == i ? kpts[3 * b + i] : 0.0,
                               &sym[(((size_t)b * 3 + i) * 3 + j) * ctx->N]);
    }
  }
  PC_CK(cudaMemcpyAsync(ctx->kparam.p, kp.data(), sizeof(KParam) * nb, cudaMemcpyHostToDevice, ctx->stream));
  PC_CK(cudaMemcpyAsync(ctx->symd.p, sym.data(), sizeof(double2) * sym.size(), cudaMemcpyHostToDevice, ctx->stream));
  PC_CK(cudaStreamSynchronize(ctx->stream));  // host staging vectors go out of scope
  return PC_OK;
}

cudaError_t get_event(pc_ctx *ctx, cudaEvent_t *e) {
  if (!ctx->event_pool.empty()) {
    *e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreate(e);
}

int harvest_timing(pc_ctx *ctx) {
  std::vector<pc_ctx::Pending> keep;
  for (auto &p : ctx->pending) {
    const cudaError_t q = cudaEventQuery(p.b);
    if (q == cudaErrorNotReady) {
      keep.push_back(p);
      continue;
    }
    PC_CK(q);
    float ms = 0.f;
    PC_CK(cudaEventElapsedTime(&ms, p.a, p.b));
    ctx->stats[p.stage].ms += ms;
    ctx->event_pool.push_back(p.a);
    ctx->event_pool.push_back(p.b);
  }
  ctx->pending.swap(keep);
  return PC_OK;
}

}  // namespace pc

using namespace pc;

extern "C" const char *pc_last_error(void) { return g_err; }

extern "C" int pc_set_timing(pc_ctx *ctx, int enable) {
  PC_REQUIRE(ctx, "pc_set_timing: null context");
  ctx->timing = enable != 0;
  return PC_OK;
}

extern "C" int pc_get_stats(pc_ctx *ctx, pc_stage_stat *out) {
  PC_REQUIRE(ctx && out, "pc_get_stats: null argument");
  PC_CK(cudaStreamSynchronize(ctx->stream));
  int rc = harvest_timing(ctx);
  if (rc) return rc;
  for (int i = 0; i < PC_NSTAGES; ++i) out[i] = ctx->stats[i];
  return PC_OK;
}

extern "C" int pc_reset_stats(pc_ctx *ctx) {
  PC_REQUIRE(ctx, "pc_reset_stats: null context");
  PC_CK(cudaStreamSynchronize(ctx->stream));
  int rc = harvest_timing(ctx);
  if (rc) return rc;
  for (int i = 0; i < PC_NSTAGES; ++i) ctx->stats[i] = pc_stage_stat{};
  return PC_OK;
}

extern "C" int pc_opts_default(pc_opts *o) {
  PC_REQUIRE(o, "pc_opts_default: null");
  std::memset(o, 0, sizeof(*o));
  o->order = 1;
  o->gamma_override = 0.0;
  o->precond = PC_PRECOND_GAMMA;
  o->precision = PC_PREC_FP64;
  o->guard = -1;
  o->maxiter = 400;
  o->max_doublings = 8;
  o->seed = 0;
  o->groups = 0;
  o->kchunk = 0;
  return PC_OK;
}

extern "C" int pc_setup(pc_ctx **out, int N, const double *eps_edges, const double *lattice, const pc_opts *opts,
                        void *stream) {
  PC_REQUIRE(out && eps_edges, "pc_setup: null argument");
  *out = nullptr;
  PC_REQUIRE(is_pow2(N) && N >= 8 && N <= 256, "pc_setup: N must be a power of two in [8, 256], got %d", N);
  // lattice[3 n + c] = component c of a_{n+1}: A = (a_1, a_2, a_3) column by column
  double amat[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, binv[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  bool general = false;
  if (lattice) {
    for (int i = 0; i < 9; ++i) {
      PC_REQUIRE(std::isfinite(lattice[i]), "pc_setup: lattice entries must be finite");
      if (lattice[i] != ((i % 4 == 0) ? 1.0 : 0.0)) general = true;
    }
    if (general && invert_lattice(lattice, amat, binv) != 0) {
      set_error("pc_setup: the lattice vectors must be linearly independent");
      return PC_EINVAL;
    }
  }
  pc_opts o;
  pc_opts_default(&o);
  if (opts) o = *opts;
  if (o.order < 1 || o.order > 4) {
    set_error("pc_setup: stencil order %d: Table 1 orders 1..4 (2nd to 8th order) are implemented", o.order);
    return PC_EUNSUPPORTED;
  }
  if (o.order > 1 && o.precision == PC_PREC_MIXED) {
    set_error("pc_setup: the mixed-precision solve implements the second-order stencils (order 1) only");
    return PC_EUNSUPPORTED;
  }
  PC_REQUIRE(o.precond == PC_PRECOND_GAMMA || o.precond == PC_PRECOND_LAPLACIAN, "pc_setup: bad precond");
  PC_REQUIRE(o.precision == PC_PREC_FP64 || o.precision == PC_PREC_MIXED, "pc_setup: bad precision");
  PC_REQUIRE(o.maxiter >= 1 && o.max_doublings >= 0, "pc_setup: bad maxiter/doublings");
  PC_REQUIRE(o.kchunk >= 0, "pc_setup: kchunk must be >= 0");
  const long n = (long)N * N * N;
  for (long i = 0; i < 3 * n; ++i)
    PC_REQUIRE(eps_edges[i] > 0.0 && std::isfinite(eps_edges[i]), "pc_setup: eps_edges[%ld] must be finite and > 0", i);

  pc_ctx *ctx = new pc_ctx();
  ctx->N = N;
  ctx->logN = ilog2(N);
  ctx->n = n;
  ctx->opts = o;
  ctx->stream = (cudaStream_t)stream;
  ctx->lat = general;
  std::memcpy(ctx->amat, amat, sizeof(amat));
  std::memcpy(ctx->binv, binv, sizeof(binv));
  std::vector<double> m0(3 * n);
  std::vector<float> m0f(3 * n);
  std::vector<float2> m0p(3 * n);  // double-float pairs of m0
  for (long i = 0; i < 3 * n; ++i) {
    m0[i] = 1.0 / eps_edges[i];
    m0f[i] = (float)m0[i];
    m0p[i] = make_float2(m0f[i], (float)(m0[i] - (double)m0f[i]));
  }
  std::vector<double2> tw(N / 2);
  std::vector<float2> twf(N / 2);
  for (int t = 0; t < N / 2; ++t) {
    const double a = -2.0 * M_PI * t / N;
    tw[t].x = std::cos(a);
    tw[t].y = std::sin(a);
    twf[t].x = (float)tw[t].x;
    twf[t].y = (float)tw[t].y;
  }
  auto fail = [&](int code) {
    delete ctx;
    return code;
  };
  cudaError_t e;
  if ((e = ctx->m0d.reserve(sizeof(double) * 3 * n)) != cudaSuccess) return fail(cuda_fail(e, "m0d", __FILE__, __LINE__));
  if ((e = ctx->m0f.reserve(sizeof(float) * 3 * n)) != cudaSuccess) return fail(cuda_fail(e, "m0f", __FILE__, __LINE__));
  if ((e = ctx->m0p.reserve(sizeof(float2) * 3 * n)) != cudaSuccess) return fail(cuda_fail(e, "m0p", __FILE__, __LINE__));
  if ((e = ctx->twd.reserve(sizeof(double2) * (N / 2))) != cudaSuccess) return fail(cuda_fail(e, "tw", __FILE__, __LINE__));
  if ((e = ctx->twf.reserve(sizeof(float2) * (N / 2))) != cudaSuccess) return fail(cuda_fail(e, "twf", __FILE__, __LINE__));
  if ((e = cudaMemcpy(ctx->m0d.p, m0.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->m0f.p, m0f.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->m0p.p, m0p.data(), sizeof(float2) * 3 * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->twd.p, tw.data(), sizeof(double2) * (N / 2), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->twf.p, twf.data(), sizeof(float2) * (N / 2), cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(cuda_fail(e, "upload", __FILE__, __LINE__));
  *out = ctx;
  return PC_OK;
}

extern "C" void pc_destroy(pc_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

namespace {

double reduce_component(double k) {
  const double g = 2.0 * M_PI;
  return k - g * std::nearbyint(k / g);
}

// Bloch vector reduced by the reciprocal lattice G = 2 pi A^{-T} n of a general cell: n = round(A^T k / 2 pi),
// k' = k - 2 pi A^{-T} n; a k whose fractional coordinates A^T k / 2 pi all lie within 1e-12 of integers is
// equivalent to 0 and becomes exactly 0
void reduce_lattice(const pc_ctx *ctx, const double *k, double *out) {
  const double g = 2.0 * M_PI;
  double f[3], nr[3];
  bool zero = true;
  for (int j = 0; j < 3; ++j) {
    f[j] = (ctx->amat[j] * k[0] + ctx->amat[3 + j] * k[1] + ctx->amat[6 + j] * k[2]) / g;  // (A^T k)_j / 2 pi
    nr[j] = std::nearbyint(f[j]);
    if (std::fabs(f[j] - nr[j]) > 1e-12) zero = false;
  }
  for (int i = 0; i < 3; ++i)
    out[i] = zero ? 0.0 : k[i] - g * (ctx->binv[i] * nr[0] + ctx->binv[3 + i] * nr[1] + ctx->binv[6 + i] * nr[2]);
}

}  // namespace

// FP64 finish of the mixed solve: the k-points it handed over (phase 2 stalled or capped) are solved again by the
// FP64 solve, started from their double-float blocks (all m columns, converted to complex128), with the same bands,
// guard columns and tolerance. Their eigenvalues, residuals and eigenvectors replace the mixed solve's; their
// iteration counts add up; ctx->fp64_finish flags them.
static int fp64_finish(pc_ctx *ctx, const double *kpts, int nbands, int m, double tol, double *evals, void *evecs,
                       int *iters, double *resid, const std::vector<std::pair<int, int>> &handover, int status) {
  const int ns = (int)handover.size(), nb = (int)ctx->fp64_finish.size();
  const long L = 3 * ctx->n;
  const size_t xcount = (size_t)ns * m * L, ecount = evecs ? (size_t)ns * nbands * L : 0;
  PC_CK(ctx->finbuf.reserve(sizeof(double2) * (xcount + ecount)));
  double2 *x0 = ctx->finbuf.as<double2>();
  double2 *ev = evecs ? x0 + xcount : nullptr;
  std::vector<double> ks(3 * (size_t)ns);
  for (int i = 0; i < ns; ++i) {
    const int b = handover[i].first, buf = handover[i].second;
    for (int d = 0; d < 3; ++d) ks[3 * i + d] = kpts[3 * b + d];
    const int rc = launch_pairs_to_c128(1, L, m, ctx->X64[buf].as<float4>() + (size_t)b * m * L, (long)m * L,
                                        x0 + (size_t)i * m * L, (long)m * L, ctx->stream, nullptr);
    if (rc) return rc;
  }
  std::vector<double> ev_s((size_t)ns * nbands), res_s((size_t)ns * nbands);
  std::vector<int> it_s(ns, 0);
  const pc_opts saved = ctx->opts;
  const void *saved_x0 = ctx->x0;
  const int saved_x0n = ctx->x0n, saved_kidx0 = ctx->kidx0;
  const bool saved_c128 = ctx->x0_c128;
  ctx->opts.precision = PC_PREC_FP64;
  ctx->opts.guard = m - nbands;
  ctx->x0 = x0;
  ctx->x0n = m;
  ctx->x0_c128 = true;
  const int rc = pc_solve(ctx, ns, ks.data(), nbands, tol, ev_s.data(), ev, it_s.data(), res_s.data());
  ctx->opts = saved;
  ctx->x0 = saved_x0;
  ctx->x0n = saved_x0n;
  ctx->kidx0 = saved_kidx0;
  ctx->x0_c128 = saved_c128;
  ctx->fp64_finish.assign(nb, 0);
  if (rc < 0) return rc;
  for (int i = 0; i < ns; ++i) {
    const int b = handover[i].first;
    for (int j = 0; j < nbands; ++j) {
      evals[(size_t)b * nbands + j] = ev_s[(size_t)i * nbands + j];
      if (resid) resid[(size_t)b * nbands + j] = res_s[(size_t)i * nbands + j];
    }
    if (iters) iters[b] += it_s[i];
    if (evecs)
      PC_CK(cudaMemcpyAsync(static_cast<double2 *>(evecs) + (size_t)b * nbands * L, ev + (size_t)i * nbands * L,
                            sizeof(double2) * (size_t)nbands * L, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->fp64_finish[b] = 1;
  }
  PC_CK(cudaStreamSynchronize(ctx->stream));
  return std::max(status, rc);
}

extern "C" int pc_solve(pc_ctx *ctx, int nk, const double *kpts, int nbands, double tol, double *evals, void *evecs,
                        int *iters, double *resid) {
  PC_REQUIRE(ctx && kpts && evals, "pc_solve: null argument");
  PC_REQUIRE(nk >= 1 && nbands >= 1, "pc_solve: need nk >= 1 and nbands >= 1");
  PC_REQUIRE(tol > 0.0 && tol < 1.0, "pc_solve: tol must be in (0, 1)");
  // guard < 0: half the bands plus one (a block that also holds the next cluster converges in ~half the
  // iterations of a tight block when clusters are cut), capped so that 3 m <= 64
  const int guard = ctx->opts.guard >= 0 ? ctx->opts.guard : std::max(0, std::min(nbands / 2 + 1, 21 - nbands));
  const int m = nbands + guard;
  PC_REQUIRE(3 * m <= 64, "pc_solve: nbands + guard must be <= 21");
  // k-points per pass that fit the device: the solve's panels take ~136 m L bytes per k-point in the mixed solve
  // (four complex64 panels of 3m columns, two double-float blocks and a complex64 residual copy) and 192 m L in the
  // FP64 solve (four complex128 panels); the two-pass stencils (general cell, orders above 1) add their scratch of
  // 4 n entries of 16 bytes per column (64 n m); the chunked reductions' partial sums add a few percent. The budget
  // is 85% of the free memory plus what this context already holds in those buffers. A batch larger than that is
  // solved in consecutive chunks; each chunk passes its offset in the caller's list, so that every k-point starts
  // from the initial block of its own index, as in an unchunked solve (the results agree to the tolerance: the
  // chunked reductions' summation order depends on the batch size).
  {
    const double Lb = 3.0 * (double)ctx->n;
    const bool two_pass = ctx->lat || ctx->opts.order > 1;
    const double per_k = 1.05 * ((ctx->opts.precision == PC_PREC_MIXED ? 136.0 : 192.0) * m * Lb +
                                 (two_pass ? 64.0 * (double)ctx->n * m : 0.0));
    size_t freeb = 0, totalb = 0;
    PC_CK(cudaMemGetInfo(&freeb, &totalb));
    double held = 0.0;
    for (int i = 0; i < 2; ++i) held += (double)ctx->S[i].bytes + (double)ctx->AS[i].bytes + (double)ctx->X64[i].bytes;
    held += (double)ctx->R32.bytes + (double)ctx->kscratch.bytes;
    for (const auto &kb : ctx->kscratch_x) held += (double)kb.bytes;
    const double budget = 0.85 * ((double)freeb + held);
    int chunk = (int)std::max(1.0, std::min(std::floor(budget / per_k), (double)nk));
    if (ctx->opts.kchunk > 0) chunk = std::min(chunk, ctx->opts.kchunk);
    if (chunk < nk) {
      int status = PC_OK;
      const void *x0 = ctx->x0;  // a caller's initial block (pc_solve_init) covers all nk k-points
      const int kidx_base = ctx->kidx0;
      const size_t x0_elem = ctx->x0_c128 ? sizeof(double2) : sizeof(float2);
      std::vector<int> finish(nk, 0);
      for (int b0 = 0; b0 < nk; b0 += chunk) {
        const int nc = std::min(chunk, nk - b0);
        ctx->kidx0 = kidx_base + b0;
        if (x0)
          ctx->x0 = static_cast<const char *>(x0) + x0_elem * (size_t)b0 * ctx->x0n * (size_t)(3 * ctx->n);
        void *ev = evecs ? static_cast<void *>(static_cast<char *>(evecs) + sizeof(double2) * (size_t)b0 * nbands *
                                                                                 (size_t)(3 * ctx->n))
                         : nullptr;
        const int rc = pc_solve(ctx, nc, kpts + 3 * (size_t)b0, nbands, tol, evals + (size_t)b0 * nbands, ev,
                                iters ? iters + b0 : nullptr, resid ? resid + (size_t)b0 * nbands : nullptr);
        ctx->x0 = x0;
        ctx->kidx0 = kidx_base;
        if (rc < 0) return rc;
        status = std::max(status, rc);
        for (int i = 0; i < nc && i < (int)ctx->fp64_finish.size(); ++i) finish[b0 + i] = ctx->fp64_finish[i];
      }
      ctx->fp64_finish = finish;
      return status;
    }
  }
  cudaStream_t st = ctx->stream;
  const int nb = nk;
  const long n = ctx->n, L = 3 * n;
  const double h = 1.0 / ctx->N;

  std::vector<double> kr(3 * nb), gam(nb);
  std::vector<int> zero(nb), doublings(nb, 0), itcount(nb, 0), done(nb, 0), round_start(nb, 0);
  for (int b = 0; b < nb; ++b) {
    double k2 = 0;
    if (ctx->lat) reduce_lattice(ctx, kpts + 3 * b, &kr[3 * b]);
    for (int d = 0; d < 3; ++d) {
      if (!ctx->lat) kr[3 * b + d] = reduce_component(kpts[3 * b + d]);
      k2 += kr[3 * b + d] * kr[3 * b + d];
    }
    zero[b] = (k2 == 0.0);
    gam[b] = ctx->opts.gamma_override > 0 ? ctx->opts.gamma_override
                                          : (k2 == 0.0 ? 2.0 / h : 2.0 * std::max(1.0 / h, 1.0 / k2));
  }
  ctx->fp64_finish.assign(nb, 0);
  int rc = upload_kpoints(ctx, nb, kr.data(), gam.data());
  if (rc) return rc;
  if (ctx->opts.precision == PC_PREC_MIXED) {
    std::vector<std::pair<int, int>> handover;
    rc = solve_mixed(ctx, nb, kr.data(), gam, zero, nbands, m, tol, evals, evecs, iters, resid, &handover);
    const int tc = gram_tc_check();  // a time-out inside the tensor-core Gram kernel voids the result
    if (tc) return tc;
    if (rc < 0 || handover.empty()) return rc;
    return fp64_finish(ctx, kpts, nbands, m, tol, evals, evecs, iters, resid, handover, rc);
  }

  const long sS = 3L * m * L;  // panel stride per k-point (elements)
  const size_t panel = sizeof(double2) * (size_t)sS * nb;
  for (int i = 0; i < 2; ++i) {
    PC_CK(ctx->S[i].reserve(panel));
    PC_CK(ctx->AS[i].reserve(panel));
  }
  const int nmax = 3 * m;
  PC_CK(ctx->Gm.reserve(sizeof(double2) * (size_t)nb * nmax * nmax));
  PC_CK(ctx->Hm.reserve(sizeof(double2) * (size_t)nb * nmax * nmax));
  PC_CK(ctx->coef.reserve(sizeof(double2) * (size_t)nb * nmax * m));
  PC_CK(ctx->theta.reserve(sizeof(double) * (size_t)nb * m));
  PC_CK(ctx->norms.reserve(sizeof(double) * (size_t)nb * m * 2));
  PC_CK(ctx->rnorm.reserve(sizeof(double) * (size_t)nb * m * 3));
  PC_CK(ctx->rank.reserve(sizeof(int) * (size_t)nb * 2));
  PC_CK(ctx->flag.reserve(sizeof(int) * (size_t)nb));
  // the chunked reductions' partial sums depend on the active count (not monotonically): size for every count
  size_t scr = 16;
  for (int na = 1; na <= nb; ++na)
    scr = std::max({scr, gram_pair_scratch_bytes(na, L, nmax), residual_scratch_bytes(na, L, m),
                    deflate_scratch_bytes(na, m), sizeof(double) * 3 * (size_t)na * m * 64});
  PC_CK(ctx->scratch.reserve(scr));
  int *d_act = ctx->rank.as<int>() + nb;
  int *d_zero = ctx->flag.as<int>();
  PC_CK(ctx->mask.reserve(sizeof(int) * (size_t)nb * m));
  int *d_mask = ctx->mask.as<int>();
  uint64_t restarts = 0;
  const bool verbose = std::getenv("PC_VERBOSE") != nullptr;  // host-side trace of the iteration (stderr)
  PC_CK(cudaMemcpyAsync(d_zero, zero.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));

  std::vector<int> act;
  for (int b = 0; b < nb; ++b) act.push_back(b);
  auto upload_act = [&]() -> int {
    PC_CK(cudaMemcpyAsync(d_act, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice, st));
    PC_CK(cudaStreamSynchronize(st));
    return PC_OK;
  };
  if ((rc = upload_act())) return rc;
  bool any_zero = false;
  for (int b = 0; b < nb; ++b) any_zero |= zero[b] != 0;

  double2 *S[2] = {ctx->S[0].as<double2>(), ctx->S[1].as<double2>()};
  double2 *AS[2] = {ctx->AS[0].as<double2>(), ctx->AS[1].as<double2>()};
  double2 *Gm = ctx->Gm.as<double2>(), *Hm = ctx->Hm.as<double2>(), *coef = ctx->coef.as<double2>();
  double *theta = ctx->theta.as<double>(), *norms = ctx->norms.as<double>(), *rn = ctx->rnorm.as<double>();
  void *scratch = ctx->scratch.p;
  const double drop = 1e-12;

#define RUN(x)                 \
  do {                         \
    int rc_ = (x);             \
    if (rc_ != PC_OK) return rc_; \
  } while (0)

  // algorithmic work per stage invocation (FP64: 16 bytes per complex entry)
  const double cb = 16.0, Ld = (double)L, nd = (double)n;
  const double op_flops = 214.0 * nd, op_bytes = 2.0 * Ld * cb;  // per field; M0 (24 B/point) once per call
  const double fft_flops = 3.0 * 2.0 * 5.0 * nd * std::log2(nd) + 60.0 * nd;
  auto OP = [&](int nbk, const void *X, void *Y) {
    return run_stage(ctx, PC_STAGE_STENCIL, 1, op_flops * nbk * m, op_bytes * nbk * m + 24.0 * nd,
                     [&] { return launch_apply_op(ctx, nbk, m, PC_C128, X, sS, Y, sS, d_act); });
  };
  auto PRE = [&](int nbk, void *R) {
    return run_stage(ctx, PC_STAGE_PRECOND, 5, fft_flops * nbk * m, 2.0 * Ld * cb * nbk * m,
                     [&] { return launch_precond(ctx, nbk, m, PC_C128, R, sS, R, sS, d_act); });
  };
  // G = S^H S and H = S^H AS, Hermitian: p (p + 1) / 2 entries each, 8 flops per complex product
  auto GRAM = [&](int nbk, int p, const void *Sx, const void *ASx) {
    return run_stage(ctx, PC_STAGE_GRAM, 2, 2.0 * 8.0 * p * (p + 1) / 2.0 * Ld * nbk, 2.0 * p * Ld * cb * nbk, [&] {
      return launch_gram_pair(nbk, L, p, PC_C128, Sx, ASx, sS, Gm, Hm, scratch, scr, st, d_act);
    });
  };
  auto RR = [&](int nbk, int nn) {
    return run_stage(ctx, PC_STAGE_RR, 1, rr_flops(nn, m) * nbk, 2.0 * nn * nn * cb * nbk,
                     [&] { return launch_rr(nbk, nn, m, Gm, Hm, drop, theta, coef, nullptr, st, d_act); });
  };
  auto UPD = [&](int nbk, int p, const void *Sx, const void *Cx, long sc, void *Y) {
    return run_stage(ctx, PC_STAGE_UPDATE, 1, 8.0 * p * m * Ld * nbk, (double)(p + m) * Ld * cb * nbk,
                     [&] { return launch_block_update(nbk, L, p, m, PC_C128, Sx, sS, Cx, sc, Y, sS, st, d_act); });
  };
  auto DEFL = [&](int nbk, void *X) {
    return run_stage(ctx, PC_STAGE_OTHER, 1, 4.0 * Ld * m * nbk, 2.0 * Ld * cb * m * nbk,
                     [&] { return launch_deflate(nbk, n, m, X, sS, d_zero, scratch, st, d_act); });
  };

  // ---- initial block and Rayleigh-Ritz on span(X0)
  int cur = 0;
  const int na0 = (int)act.size();
  RUN(run_stage(ctx, PC_STAGE_OTHER, 1, 0.0, Ld * cb * m * nb,
                [&] { return launch_init_block(nb, L, m, ctx->opts.seed, ctx->kidx0, S[0], sS, st); }));
  if (ctx->x0) RUN(launch_copy_x0(ctx, 0, nb, PC_C128, S[0], sS, st));
  if (any_zero) RUN(DEFL(na0, S[0]));
  RUN(OP(na0, S[0], AS[0]));
  RUN(GRAM(na0, m, S[0], AS[0]));
  RUN(RR(na0, m));
  RUN(UPD(na0, m, S[0], coef, (long)m * m, S[1]));
  RUN(OP(na0, S[1], AS[1]));
  cur = 1;
  bool haveP = false;

  std::vector<double> h_theta((size_t)nb * m), h_norms((size_t)nb * m * 2), h_rn((size_t)nb * m * 3);
  int status = PC_OK;
  const int maxiter = ctx->opts.maxiter;
  for (int it = 0;; ++it) {
    const int na = (int)act.size();
    double2 *Sc = S[cur], *ASc = AS[cur];
    // residual into the W slot
    RUN(run_stage(ctx, PC_STAGE_RESIDUAL, 2, 8.0 * Ld * m * na, 3.0 * Ld * cb * m * na, [&] {
      return launch_residual(na, L, m, Sc, sS, ASc, sS, theta, Sc + (long)m * L, sS, norms, scratch, scr, st, d_act);
    }));
    PC_CK(cudaMemcpyAsync(h_theta.data(), theta, sizeof(double) * nb * m, cudaMemcpyDeviceToHost, st));
    PC_CK(cudaMemcpyAsync(h_norms.data(), norms, sizeof(double) * nb * m * 2, cudaMemcpyDeviceToHost, st));
    PC_CK(cudaStreamSynchronize(st));
    if ((rc = harvest_timing(ctx))) return rc;
    if (verbose) {
      for (int b : act) {
        double mx = 0;
        for (int j = 0; j < nbands; ++j) {
          const double r = h_norms[((size_t)b * m + j) * 2], x = h_norms[((size_t)b * m + j) * 2 + 1];
          mx = std::max(mx, r / (std::fabs(h_theta[(size_t)b * m + j]) * x));
        }
        std::fprintf(stderr, "[pc] it %d k %d gamma %.4g maxres %.3e theta0..%d = %.6g .. %.6g\n", it, b, gam[b], mx,
                     m - 1, h_theta[(size_t)b * m], h_theta[(size_t)b * m + m - 1]);
      }
    }
    std::vector<int> conv;
    for (int b : act) {
      bool ok = true;
      for (int j = 0; j < nbands; ++j) {
        const double r = h_norms[((size_t)b * m + j) * 2], x = h_norms[((size_t)b * m + j) * 2 + 1];
        if (!(r <= tol * std::fabs(h_theta[(size_t)b * m + j]) * x)) ok = false;
      }
      if (ok || it - round_start[b] >= maxiter) conv.push_back(b);
    }
    // Algorithm 4.1 on the k-points that just converged
    std::vector<int> redo, fin;
    if (!conv.empty()) {
      PC_CK(cudaMemcpyAsync(d_act, conv.data(), sizeof(int) * conv.size(), cudaMemcpyHostToDevice, st));
      const int nconv = (int)conv.size();
      RUN(run_stage(ctx, PC_STAGE_RECOMPUTE, 2, 120.0 * nd * m * nconv, Ld * cb * m * nconv,
                    [&] { return launch_recompute(ctx, nconv, m, Sc, sS, rn, d_act, scratch, scr); }));
      PC_CK(cudaMemcpyAsync(h_rn.data(), rn, sizeof(double) * nb * m * 3, cudaMemcpyDeviceToHost, st));
      PC_CK(cudaStreamSynchronize(st));
      for (int b : conv) {
        bool spurious = false;
        for (int j = 0; j < nbands; ++j) {
          const double *o = &h_rn[((size_t)b * m + j) * 3];
          const double lre = o[0] / o[2], lam = h_theta[(size_t)b * m + j];
          if (std::fabs(lam - lre) > 10.0 * tol * std::fabs(lam)) spurious = true;
        }
        const bool capped = it - round_start[b] >= maxiter;
        if (spurious && doublings[b] < ctx->opts.max_doublings && !capped) {
          redo.push_back(b);
        } else {
          if (spurious) status = std::max(status, PC_SPURIOUS);
          if (capped) status = std::max(status, PC_NOT_CONVERGED);
          fin.push_back(b);
        }
      }
    }
    for (int b : fin) {
      done[b] = 1;
      itcount[b] = it;
      for (int j = 0; j < nbands; ++j) {
        evals[(size_t)b * nbands + j] = h_theta[(size_t)b * m + j];
        if (resid) {
          const double r = h_norms[((size_t)b * m + j) * 2], x = h_norms[((size_t)b * m + j) * 2 + 1];
          resid[(size_t)b * nbands + j] = r / (std::fabs(h_theta[(size_t)b * m + j]) * x);
        }
      }
      if (evecs)
        PC_CK(cudaMemcpyAsync(static_cast<double2 *>(evecs) + (size_t)b * nbands * L, Sc + (size_t)b * sS,
                              sizeof(double2) * (size_t)nbands * L, cudaMemcpyDeviceToDevice, st));
    }
    {
      std::vector<int> keep;
      for (int b : act)
        if (!done[b]) keep.push_back(b);
      act.swap(keep);
    }
    if (act.empty()) break;
    if (!redo.empty()) {
      // gamma doubling (Algorithm 4.1): refresh parameters, recompute AX (and AP) for those k-points
      for (int b : redo) {
        gam[b] *= 2.0;
        doublings[b] += 1;
        round_start[b] = it + 1;
      }
      RUN(upload_kpoints(ctx, nb, kr.data(), gam.data()));
      PC_CK(cudaMemcpyAsync(d_act, redo.data(), sizeof(int) * redo.size(), cudaMemcpyHostToDevice, st));
      // "goto line 1" warm-started: spurious columns are exact gamma-independent eigenvectors of B'B that LOBPCG
      // would never leave; they are replaced by fresh counter-based columns before the re-solve
      std::vector<int> mask((size_t)nb * m);
      spurious_mask(redo, m, nbands, tol, h_theta, h_rn, mask);
      if (verbose)
        for (int b : redo) {
          std::fprintf(stderr, "[pc] it %d k %d doubling -> gamma %.4g, replaced columns:", it, b, gam[b]);
          for (int j = 0; j < m; ++j)
            if (mask[(size_t)b * m + j]) std::fprintf(stderr, " %d", j);
          std::fprintf(stderr, "\n");
        }
      PC_CK(cudaMemcpyAsync(d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, st));
      ++restarts;
      RUN(run_stage(ctx, PC_STAGE_OTHER, 1, 0.0, 0.0, [&] {
        return launch_init_block((int)redo.size(), L, m, ctx->opts.seed + 7919ULL * restarts, 0, Sc, sS, st, d_mask,
                                 d_act);
      }));
      if (any_zero) RUN(DEFL((int)redo.size(), Sc));
      RUN(OP((int)redo.size(), Sc, ASc));
      if (haveP)
        RUN(OP((int)redo.size(), Sc + 2L * m * L, ASc + 2L * m * L));
      if ((rc = upload_act())) return rc;
      continue;  // recompute residuals with the new operator
    }
    if ((rc = upload_act())) return rc;
    const int nc = haveP ? 3 * m : 2 * m;
    const int na2 = (int)act.size();
    const int nxt = 1 - cur;
    double2 *Sn = S[nxt], *ASn = AS[nxt];
    // W = P^{-1} R, AW = Op W
    RUN(PRE(na2, Sc + (long)m * L));
    if (any_zero) RUN(DEFL(na2, Sc + (long)m * L));
    RUN(OP(na2, Sc + (long)m * L, ASc + (long)m * L));
    // Rayleigh-Ritz on span[X W P]
    RUN(GRAM(na2, nc, Sc, ASc));
    RUN(RR(na2, nc));
    // X' = S coef, P' = [W P] coef_{W,P}
    RUN(UPD(na2, nc, Sc, coef, (long)nc * m, Sn));
    RUN(UPD(na2, nc - m, Sc + (long)m * L, coef + (long)m * m, (long)nc * m, Sn + 2L * m * L));
    if (any_zero) {
      RUN(DEFL(na2, Sn));
      RUN(DEFL(na2, Sn + 2L * m * L));
    }
    RUN(OP(na2, Sn, ASn));
    RUN(OP(na2, Sn + 2L * m * L, ASn + 2L * m * L));
    cur = nxt;
    haveP = true;
  }
#undef RUN
  PC_CK(cudaStreamSynchronize(st));
  if (iters)
    for (int b = 0; b < nb; ++b) iters[b] = itcount[b];
  return status;
}

extern "C" int pc_get_fp64_finish(pc_ctx *ctx, int nk, int *flags) {
  PC_REQUIRE(ctx && flags, "pc_get_fp64_finish: null argument");
  PC_REQUIRE(nk == (int)ctx->fp64_finish.size(), "pc_get_fp64_finish: nk differs from the last solve's");
  for (int b = 0; b < nk; ++b) flags[b] = ctx->fp64_finish[b];
  return PC_OK;
}

extern "C" int pc_solve_init(pc_ctx *ctx, int nk, const double *kpts, int nbands, double tol, const void *X0, int n0,
                             double *evals, void *evecs, int *iters, double *resid) {
  PC_REQUIRE(ctx && X0, "pc_solve_init: null argument");
  PC_REQUIRE(n0 >= 1 && n0 <= nbands, "pc_solve_init: need 1 <= n0 <= nbands, got n0 = %d", n0);
  ctx->x0 = X0;
  ctx->x0n = n0;
  const int rc = pc_solve(ctx, nk, kpts, nbands, tol, evals, evecs, iters, resid);
  ctx->x0 = nullptr;
  ctx->x0n = 0;
  return rc;
}
