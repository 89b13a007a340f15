// Mixed-precision batched LOBPCG (PC_PREC_MIXED): the search directions W, P, their operator images and every
// tall-skinny product over them run in complex64; the block X, its image AX, the residual and the X-X block of the
// Rayleigh-Ritz pencil are FP64 once the complex64 iteration has stopped improving; the small Rayleigh-Ritz
// eigenproblem is always FP64 (Section 5.1's LOBPCG with the preconditioner of Section 5.2).
//
// Two numerical facts shape it:
// * The X-Q coupling of the projected operator, X^H Op Q, must not be formed as X^H (Op Q) in complex64: Op Q is
//   |Op| |Q| large while the coupling is O(|R| |Q|), so the rounding of the product swamps it. Because Op is Hermitian
//   and AX = X Theta + R exactly (R is defined that way), X^H Op Q = Theta X^H Q + R^H Q, which only multiplies
//   small, accurately stored quantities.
// * The X-X block (X^H X, X^H AX) and the residual need FP64: the residual floor of a complex64 X is
//   eps32 |Op| / lambda (about 1e-3 here), and the X-X block's rounding shifts the Ritz values by eps32 lambda.
// Phase 1 (every k-point starts here): X and AX in complex64 as well, until the complex64 residual stops falling.
// Phase 2: X stored as double-float pairs (hi + lo FP32, ~48 bits); X' = X C_X + P' (complex64 correction),
// AX' = Op X' by the stencil fused with the residual R = AX' - X' Theta (AX' itself is never stored), and the X-X
// Gram block X^H X, all three in double-float arithmetic (mixed_df.cu) on the FP32 pipe. The X-X block of the
// projected operator is Theta X^H X + R^H X (AX = X Theta + R), with R^H X from the complex64 product R^H [X | Q]:
// its rounding is eps32 |R| |X|, small because R is.
// Convergence and Algorithm 4.1 are decided in phase 2 only, on FP64 residuals and FP64 norms. A k-point whose
// phase 2 stops converging (its largest residual below 1e-2 and its best over the last 25 iterations not 20% below
// the best of the 25 before, after at least 50), jumps (1000 times above its best, handed over with the block of
// the iteration before), or reaches maxiter is handed back unfinished: pc_solve finishes it with the FP64 solve from its double-float block.
// (Measured at N = 128 near Gamma, where the lowest bands have lambda ~ 0.09: their phase 2 levels off at a
// relative residual of 1e-5 to 1e-4 -- an absolute residual of ~1e-6 |x|, as for every other band there -- while
// the FP64 solve reaches the tolerance.)
//
// Scheduling: the k-points are split into contiguous groups (opts.groups, up to 4; default 4 from 16 k-points, 2
// from 8), each with its own stream, active list, scratch and pinned host copies of its residual norms. Every
// iteration of a group ends with its residual norms copied to the host and an event; the host then serves the
// groups in turn -- waits for a group's event, takes its convergence decisions, enqueues its next iteration -- so
// that while it waits for one group the other groups' kernels occupy the GPU. This hides the latency-bound steps (the Rayleigh-Ritz
// kernel runs one block per k-point, the host decisions leave the GPU idle) behind bandwidth-bound kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <utility>
#include <vector>

#include "pc_internal.cuh"
#include "phase_rules.h"

namespace pc {

namespace {

#define RUN(x)                    \
  do {                            \
    int rc_ = (x);                \
    if (rc_ != PC_OK) return rc_; \
  } while (0)

// state shared by the groups of one solve (per-k-point arrays are indexed by the global k-point index b)
struct MixedShared {
  pc_ctx *ctx;
  int nb, nbands, m;
  long n, L, sF, sX;
  int nmax;
  double tol, drop;
  const double *kr;
  std::vector<double> *gam;
  bool any_zero;
  std::vector<int> zero;  // per k-point: k reduced to 0 (the constant fields are projected out)
  float2 *F[2], *AF[2];
  float4 *X64[2];  // phase-2 block, double-float pairs (PC_DFS)
  float2 *R32;
  double2 *Gm, *Hm, *coef, *RQ, *GX;
  double *theta, *norms, *rn;
  int *d_zero, *d_phase, *d_mask;
  double *h_theta, *h_norms, *h_rn;  // pinned
  size_t scr;                        // scratch bytes per group
  // batch strides (elements) of the per-k-point matrices, fixed for every search-space width so that groups at
  // different iterations never overlap: G and H (nmax x nmax), R^H S (m x nmax), coefficients (nmax x m)
  long sG, sRS, sC;
  std::vector<int> phase, doublings, itcount, done, round_start, p1_start;
  std::vector<ResidHistory> hist;   // per k-point: (iteration, largest relative residual)
  std::vector<ResidHistory> hist2;  // the same in phase 2, since the last switch or restart
  std::vector<std::pair<int, int>> *handover = nullptr;   // unfinished k-points and the X64 buffer of their block
  Phase1Rule p1_rule;  // phase switch thresholds (phase_rules.h)
  double *evals, *resid;
  void *evecs;
  int status = PC_OK;
  double Ld, nd, fft_flops;
  int verbose = 0;  // host-side trace of the iteration (stderr): PC_VERBOSE = 1 (largest residual), 2 (every column)
};

struct Group {
  int b0 = 0, b1 = 0;  // k-points [b0, b1)
  cudaStream_t st = nullptr;
  int *d_act = nullptr;
  void *scratch = nullptr;
  std::vector<int> act;
  int cur = 1, it = 0;
  bool haveP = false, finished = false;
  uint64_t restarts = 0;
  cudaEvent_t ev = nullptr;
  cudaStream_t rst = nullptr;                        // high-priority stream of its Rayleigh-Ritz launches
  cudaEvent_t to_rr = nullptr, from_rr = nullptr;  // hand-offs between st and rst
};

class MixedSolve {
 public:
  MixedSolve(MixedShared &s, Group &g) : S(s), g(g), ctx(s.ctx) {}

  // kernels of this group go to its stream (run_stage records its events on ctx->stream)
  struct StreamScope {
    pc_ctx *ctx;
    cudaStream_t saved;
    StreamScope(pc_ctx *c, cudaStream_t s) : ctx(c), saved(c->stream) { c->stream = s; }
    ~StreamScope() { ctx->stream = saved; }
  };

  int set_act(const std::vector<int> &v) {
    if (v.empty()) return PC_OK;
    PC_CK(cudaMemcpyAsync(g.d_act, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, g.st));
    return PC_OK;
  }
  int OP32(int nbk, int cols, const void *X, long sx, void *Y, long sy) {
    return run_stage(ctx, PC_STAGE_STENCIL, 1, 214.0 * S.nd * nbk * cols, 2.0 * S.Ld * 8.0 * nbk * cols + 12.0 * S.nd,
                     [&] { return launch_apply_op(ctx, nbk, cols, PC_C64, X, sx, Y, sy, g.d_act); });
  }
  // phase 2: AX = Op X for the FP64 block in double-float arithmetic, fused with the residual R = AX - X Theta
  // (complex64 copies of R into the W slot of panel `slot` and into R32, of X and AX into the panel's X columns;
  // column norms into `norms`): the FP64 AX is never stored
  int OP64R(int nbk, const void *X, int slot) {
    const long L = S.L, sF = S.sF;
    return run_stage(ctx, PC_STAGE_DFLOAT, 2, (214.0 * S.nd + 4.0 * S.Ld) * nbk * S.m,
                     (16.0 + 4.0 * 8.0) * S.Ld * nbk * S.m + 24.0 * S.nd, [&] {
                       return launch_op_df_resid(ctx, nbk, S.m, X, S.sX, S.theta, S.F[slot] + (long)S.m * L, sF,
                                                 S.R32, S.sX, S.F[slot], sF, S.AF[slot], sF, S.norms, g.scratch, S.scr,
                                                 g.d_act);
                     });
  }
  // Rayleigh-Ritz of the group's pencils (nc columns; patch: the coupling blocks first) on the group's high-priority
  // stream, joined back to its stream: the few blocks of this latency-bound kernel then take SMs ahead of the other
  // groups' pending blocks instead of queueing behind them
  int RR(int na, int nc, bool patch) {
    const int m = S.m;
    return run_stage(ctx, PC_STAGE_RR, patch ? 2 : 1, rr_flops(nc, m) * na, 2.0 * nc * nc * 16.0 * na, [&] {
      PC_CK(cudaEventRecord(g.to_rr, g.st));
      PC_CK(cudaStreamWaitEvent(g.rst, g.to_rr, 0));
      int rc = patch ? launch_rr_patch(na, nc, m, S.Gm, S.Hm, S.RQ, S.theta, S.GX, S.d_phase, g.rst, g.d_act, S.sG,
                                       S.sRS)
                     : PC_OK;
      if (rc == PC_OK)
        rc = launch_rr(na, nc, m, S.Gm, S.Hm, S.drop, S.theta, S.coef, nullptr, g.rst, g.d_act, S.sG, S.sC);
      PC_CK(cudaEventRecord(g.from_rr, g.rst));
      PC_CK(cudaStreamWaitEvent(g.st, g.from_rr, 0));
      return rc;
    });
  }
  // projection of the constant fields on the k = 0 points of `list`, which is the active list already on the device
  // (the kernel's blocks of other k-points return at once); nothing is launched when `list` holds no k = 0 point
  int DEFL(const std::vector<int> &list, void *X, long sx, int dtype) {
    if (!S.any_zero) return PC_OK;
    int nz = 0;
    for (int b : list) nz += S.zero[b] != 0;
    if (nz == 0) return PC_OK;
    const int na = (int)list.size();
    return run_stage(ctx, PC_STAGE_OTHER, 1, 4.0 * S.Ld * S.m * nz,
                     2.0 * S.Ld * (dtype == PC_C64 ? 8.0 : 16.0) * S.m * nz,
                     [&] { return launch_deflate(na, S.n, S.m, X, sx, S.d_zero, g.scratch, g.st, g.d_act, dtype); });
  }

  // initial block (the counter-based generator, complex64) and Rayleigh-Ritz on span(X0), then the first residual
  int start() {
    StreamScope scope(ctx, g.st);
    const int m = S.m, nb = S.nb;
    const long L = S.L, sF = S.sF, sX = S.sX;
    const int na = g.b1 - g.b0;
    for (int b = g.b0; b < g.b1; ++b) g.act.push_back(b);
    RUN(set_act(g.act));
    RUN(run_stage(ctx, PC_STAGE_OTHER, 1, 0.0, S.Ld * 8.0 * m * na, [&] {
      return launch_init_block(na, L, m, ctx->opts.seed, ctx->kidx0, S.F[0], sF, g.st, nullptr, g.d_act, PC_C64);
    }));
    if (ctx->x0) RUN(launch_copy_x0(ctx, g.b0, na, PC_C64, S.F[0], sF, g.st));
    RUN(DEFL(g.act, S.F[0], sF, PC_C64));
    RUN(OP32(na, m, S.F[0], sF, S.AF[0], sF));
    RUN(run_stage(ctx, PC_STAGE_GRAM, 2, 8.0 * m * (m + 1) * S.Ld * na, 2.0 * m * S.Ld * 8.0 * na, [&] {
      return launch_gram_pair(na, L, m, PC_C64, S.F[0], S.AF[0], sF, S.Gm, S.Hm, g.scratch, S.scr, g.st, g.d_act, nb,
                              S.sG);
    }));
    RUN(RR(na, m, false));
    RUN(run_stage(ctx, PC_STAGE_UPDATE, 1, 8.0 * m * m * S.Ld * na, 2.0 * m * S.Ld * 8.0 * na, [&] {
      return launch_block_update(na, L, m, m, PC_C64, S.F[0], sF, S.coef, S.sC, S.F[1], sF, g.st, g.d_act);
    }));
    RUN(OP32(na, m, S.F[1], sF, S.AF[1], sF));
    g.cur = 1;
    g.haveP = false;
    g.it = 0;
    return residual();
  }

  // residuals of the phase-1 k-points (complex64 block), then norms and Ritz values of the group to the host and the
  // group's event
  int residual() {
    StreamScope scope(ctx, g.st);
    const int m = S.m;
    const long L = S.L, sF = S.sF, sX = S.sX;
    std::vector<int> act1, act2;
    for (int b : g.act) (S.phase[b] == 1 ? act1 : act2).push_back(b);
    const int cur = g.cur;
    if (!act1.empty()) {
      RUN(set_act(act1));
      const int na = (int)act1.size();
      RUN(run_stage(ctx, PC_STAGE_RESIDUAL, 2, 8.0 * S.Ld * m * na, 4.0 * S.Ld * 8.0 * m * na, [&] {
        return launch_residual_mixed(na, L, m, PC_C64, S.F[cur], sF, S.AF[cur], sF, S.theta, S.F[cur] + (long)m * L,
                                     sF, S.R32, sX, nullptr, 0, nullptr, 0, S.norms, g.scratch, S.scr, g.st, g.d_act);
      }));
    }
    // phase-2 residuals were produced by the fused stencil (OP64R) when their block last changed
    const size_t k0 = (size_t)g.b0 * m, kn = (size_t)(g.b1 - g.b0) * m;
    PC_CK(cudaMemcpyAsync(S.h_theta + k0, S.theta + k0, sizeof(double) * kn, cudaMemcpyDeviceToHost, g.st));
    PC_CK(cudaMemcpyAsync(S.h_norms + 2 * k0, S.norms + 2 * k0, sizeof(double) * 2 * kn, cudaMemcpyDeviceToHost,
                          g.st));
    PC_CK(cudaEventRecord(g.ev, g.st));
    return PC_OK;
  }

  double relres(int b, int j) const {
    const double r = S.h_norms[((size_t)b * S.m + j) * 2], x = S.h_norms[((size_t)b * S.m + j) * 2 + 1];
    return r / (std::fabs(S.h_theta[(size_t)b * S.m + j]) * x);
  }

  // after the group's event: decisions on its residuals, then its next iteration up to the next residual
  int step() {
    StreamScope scope(ctx, g.st);
    const int m = S.m, nb = S.nb, nbands = S.nbands;
    const long L = S.L, sF = S.sF, sX = S.sX;
    const int it = g.it, cur = g.cur, maxiter = ctx->opts.maxiter;
    std::vector<int> act1, act2;
    for (int b : g.act) (S.phase[b] == 1 ? act1 : act2).push_back(b);
    if (S.verbose)
      for (int b : g.act) {
        double mx = 0;
        for (int j = 0; j < nbands; ++j) mx = std::max(mx, relres(b, j));
        std::fprintf(stderr, "[pc-mixed] it %d k %d phase %d maxres %.3e", it, b, S.phase[b], mx);
        if (S.verbose > 1)
          for (int j = 0; j < S.m; ++j) std::fprintf(stderr, " %.2e", relres(b, j));
        std::fprintf(stderr, "\n");
      }
    // ---- phase 1 -> 2 once the complex64 residual stops falling, at its floor (phase_rules.h). The floor is eps32
    // times the stencil's magnitude (~gamma / h^2) over lambda: ~3e-3 for most k-points of a path at N = 32 and
    // ~3e-2 at N = 64, but near Gamma, where the lowest bands have small lambda (~|k|^2 / eps), it reaches 1 and
    // above (near Gamma at N = 64 the complex64 residual sits at ~2 from iteration ~20 on; without the long-stall
    // rule those k-points waited for the 150-iteration cap).
    std::vector<int> sw;
    for (int b : act1) {
      double mx = 0;
      for (int j = 0; j < nbands; ++j) mx = std::max(mx, relres(b, j));
      if (!(mx == mx)) mx = 1e300;  // NaN guard
      record_residual(S.hist[b], it, mx);
      if (phase1_done(S.hist[b], mx, it - S.p1_start[b], S.p1_rule)) sw.push_back(b);
    }
    // ---- phase 2: convergence on FP64 residuals, then Algorithm 4.1; a stalled or capped k-point is handed over
    std::vector<int> conv, hand, rollback;
    for (int b : act2) {
      bool ok = true;
      double mx = 0;
      for (int j = 0; j < nbands; ++j) {
        const double r = relres(b, j);
        if (!(r <= S.tol)) ok = false;
        mx = std::max(mx, r == r ? r : 1e300);
      }
      // a rollback hands over the block of the previous iteration, still in the other buffer (excursions up to
      // ~150x on the diamond-air-N64 batch recover by themselves; the rule waits for 1000x)
      record_residual(S.hist2[b], it, mx);
      switch (phase2_step(S.hist2[b], it, ok, mx, it - S.round_start[b] >= maxiter)) {
        case Phase2Step::kConverged: conv.push_back(b); break;
        case Phase2Step::kRollback: rollback.push_back(b); break;
        case Phase2Step::kHandover: hand.push_back(b); break;
        case Phase2Step::kContinue: break;
      }
    }
    for (int b : rollback) hand.push_back(b);
    for (int b : hand) {
      S.done[b] = 1;
      S.itcount[b] = it;
      for (int j = 0; j < nbands; ++j) {
        S.evals[(size_t)b * nbands + j] = S.h_theta[(size_t)b * m + j];
        if (S.resid) S.resid[(size_t)b * nbands + j] = relres(b, j);
      }
      const bool back = std::find(rollback.begin(), rollback.end(), b) != rollback.end();
      S.handover->push_back({b, back ? 1 - cur : cur});
      if (S.verbose)
        std::fprintf(stderr, "[pc-mixed] it %d k %d handed to the FP64 solve%s\n", it, b,
                     back ? " (previous block, after a jump)" : "");
    }
    std::vector<int> redo, fin;
    if (!conv.empty()) {
      RUN(set_act(conv));
      const int nc = (int)conv.size();
      RUN(run_stage(ctx, PC_STAGE_RECOMPUTE, 2, 120.0 * S.nd * m * nc, S.Ld * 16.0 * m * nc, [&] {
        return launch_recompute(ctx, nc, m, S.X64[cur], sX, S.rn, g.d_act, g.scratch, S.scr, PC_DFS);
      }));
      const size_t k0 = (size_t)g.b0 * m, kn = (size_t)(g.b1 - g.b0) * m;
      PC_CK(cudaMemcpyAsync(S.h_rn + 3 * k0, S.rn + 3 * k0, sizeof(double) * 3 * kn, cudaMemcpyDeviceToHost, g.st));
      PC_CK(cudaStreamSynchronize(g.st));
      for (int b : conv) {
        bool spurious = false;
        for (int j = 0; j < nbands; ++j) {
          const double *o = &S.h_rn[((size_t)b * m + j) * 3];
          const double lre = o[0] / o[2], lam = S.h_theta[(size_t)b * m + j];
          if (std::fabs(lam - lre) > 10.0 * S.tol * std::fabs(lam)) spurious = true;
        }
        const bool capped = it - S.round_start[b] >= maxiter;
        if (spurious && S.doublings[b] < ctx->opts.max_doublings && !capped) {
          redo.push_back(b);
        } else {
          if (spurious) S.status = std::max(S.status, (int)PC_SPURIOUS);
          if (capped) S.status = std::max(S.status, (int)PC_NOT_CONVERGED);
          fin.push_back(b);
        }
      }
    }
    for (int b : fin) {
      S.done[b] = 1;
      S.itcount[b] = it;
      for (int j = 0; j < nbands; ++j) {
        S.evals[(size_t)b * nbands + j] = S.h_theta[(size_t)b * m + j];
        if (S.resid) S.resid[(size_t)b * nbands + j] = relres(b, j);
      }
    }
    if (S.evecs && !fin.empty()) {
      // the first nbands columns, converted to complex128, into the caller's [nb][nbands][L] block
      RUN(set_act(fin));
      RUN(run_stage(ctx, PC_STAGE_OTHER, 1, 0.0, S.Ld * 32.0 * nbands * fin.size(), [&] {
        return launch_pairs_to_c128((int)fin.size(), L, nbands, S.X64[cur], sX, S.evecs, (long)nbands * L, g.st,
                                    g.d_act);
      }));
    }
    {
      std::vector<int> keep;
      for (int b : g.act)
        if (!S.done[b]) keep.push_back(b);
      g.act.swap(keep);
    }
    if (g.act.empty()) {
      g.finished = true;
      return PC_OK;
    }
    const int k0 = g.b0, kn = g.b1 - g.b0;
    if (!sw.empty() || !redo.empty()) {
      // phase switch: X64 = X (widened) and its residual; gamma doubling: the residual and AP with the new gamma
      if (!sw.empty()) {
        for (int b : sw) {
          S.phase[b] = 2;
          S.round_start[b] = it + 1;
          S.hist2[b].clear();
        }
        RUN(set_act(sw));
        const int ns = (int)sw.size();
        RUN(run_stage(ctx, PC_STAGE_OTHER, 1, 0.0, S.Ld * 24.0 * m * ns,
                      [&] { return launch_widen(ns, L, m, S.F[cur], sF, S.X64[cur], sX, g.st, g.d_act); }));
        RUN(OP64R(ns, S.X64[cur], cur));
        PC_CK(cudaMemcpyAsync(S.d_phase + k0, S.phase.data() + k0, sizeof(int) * kn, cudaMemcpyHostToDevice, g.st));
      }
      if (!redo.empty()) {
        for (int b : redo) {
          (*S.gam)[b] *= 2.0;
          S.doublings[b] += 1;
          S.round_start[b] = it + 1;
          S.hist2[b].clear();
        }
        RUN(upload_kpoints(ctx, nb, S.kr, S.gam->data()));
        RUN(set_act(redo));
        const int nr = (int)redo.size();
        // spurious columns (gamma-independent exact eigenvectors of B'B) are replaced by fresh random columns
        std::vector<double> th(S.h_theta, S.h_theta + (size_t)nb * m), rr(S.h_rn, S.h_rn + (size_t)nb * m * 3);
        std::vector<int> mask((size_t)nb * m);
        spurious_mask(redo, m, nbands, S.tol, th, rr, mask);
        PC_CK(cudaMemcpyAsync(S.d_mask + (size_t)k0 * m, mask.data() + (size_t)k0 * m, sizeof(int) * kn * m,
                              cudaMemcpyHostToDevice, g.st));
        ++g.restarts;
        // streams of fresh columns: distinct per group and restart
        const uint64_t seed = ctx->opts.seed + 7919ULL * (g.restarts + 1000ULL * (uint64_t)g.b0);
        RUN(run_stage(ctx, PC_STAGE_OTHER, 1, 0.0, 0.0, [&] {
          return launch_init_block(nr, L, m, seed, 0, S.X64[cur], sX, g.st, S.d_mask, g.d_act, PC_DFS);
        }));
        RUN(DEFL(redo, S.X64[cur], sX, PC_DFS));
        RUN(OP64R(nr, S.X64[cur], cur));
        if (g.haveP) RUN(OP32(nr, m, S.F[cur] + 2L * m * L, sF, S.AF[cur] + 2L * m * L, sF));
      }
      return residual();  // residuals again with the new block or operator
    }
    const int nc = g.haveP ? 3 * m : 2 * m;
    const int nq = nc - m;
    RUN(set_act(g.act));
    const int na = (int)g.act.size();
    const int nxt = 1 - cur;
    // ---- W = P^{-1} R (complex64), AW = Op W
    RUN(run_stage(ctx, PC_STAGE_PRECOND, 5, S.fft_flops * na * m, 2.0 * S.Ld * 8.0 * na * m, [&] {
      return launch_precond(ctx, na, m, PC_C64, S.F[cur] + (long)m * L, sF, S.F[cur] + (long)m * L, sF, g.d_act);
    }));
    RUN(DEFL(g.act, S.F[cur] + (long)m * L, sF, PC_C64));
    RUN(OP32(na, m, S.F[cur] + (long)m * L, sF, S.AF[cur] + (long)m * L, sF));
    // ---- pencil: complex64 products over [X | W | P] and, in the same pass, R^H [X | Q] (the coupling R^H Q of H,
    // and R^H X for the X-X block in phase 2); FP64 X-X block in phase 2
    RUN(run_stage(ctx, PC_STAGE_GRAM, 3, 8.0 * (nc * (nc + 1) + m * nc) * S.Ld * na,
                  (2.0 * nc + m) * S.Ld * 8.0 * na, [&] {
                    return launch_gram_pair_coupled(na, L, nc, m, PC_C64, S.F[cur], S.AF[cur], sF, S.R32, sX, S.Gm,
                                                    S.Hm, S.RQ, g.scratch, S.scr, g.st, g.d_act, nb, S.sG, S.sRS);
                  }));
    act1.clear();
    act2.clear();
    for (int b : g.act) (S.phase[b] == 1 ? act1 : act2).push_back(b);
    if (!act2.empty()) {
      RUN(set_act(act2));
      const int n2 = (int)act2.size();
      RUN(run_stage(ctx, PC_STAGE_DFLOAT, 2, 4.0 * m * (m + 1) * S.Ld * n2, m * S.Ld * 16.0 * n2, [&] {
        return launch_gram_df(n2, L, m, S.X64[cur], sX, S.GX, g.scratch, S.scr, g.st, g.d_act);
      }));
      RUN(set_act(g.act));
    }
    RUN(RR(na, nc, true));
    // ---- P' = [W P] coef_{W,P} (complex64), then X' per phase
    RUN(run_stage(ctx, PC_STAGE_UPDATE, 1, 8.0 * nq * m * S.Ld * na, (double)(nq + m) * S.Ld * 8.0 * na, [&] {
      return launch_block_update(na, L, nq, m, PC_C64, S.F[cur] + (long)m * L, sF, S.coef + (long)m * m, S.sC,
                                 S.F[nxt] + 2L * m * L, sF, g.st, g.d_act);
    }));
    if (!act1.empty()) {
      RUN(set_act(act1));
      const int n1 = (int)act1.size();
      // X' = X C_X + P' (the P' just formed is [W P] C_{W,P}): reads 2m columns instead of the 3m of [X W P]
      RUN(run_stage(ctx, PC_STAGE_UPDATE, 1, 8.0 * m * m * S.Ld * n1, 3.0 * m * S.Ld * 8.0 * n1, [&] {
        return launch_block_update(n1, L, m, m, PC_C64, S.F[cur], sF, S.coef, S.sC, S.F[nxt], sF, g.st, g.d_act,
                                   S.F[nxt] + 2L * m * L, sF);
      }));
      RUN(DEFL(act1, S.F[nxt], sF, PC_C64));
      RUN(OP32(n1, m, S.F[nxt], sF, S.AF[nxt], sF));
    }
    if (!act2.empty()) {
      RUN(set_act(act2));
      const int n2 = (int)act2.size();
      RUN(run_stage(ctx, PC_STAGE_DFLOAT, 1, 8.0 * m * m * S.Ld * n2, (2.0 * 16.0 + 8.0) * m * S.Ld * n2, [&] {
        return launch_update_df(n2, L, m, m, S.X64[cur], sX, S.coef, S.sC, S.X64[nxt], sX,
                                S.F[nxt] + 2L * m * L, sF, g.st, g.d_act);
      }));
      RUN(DEFL(act2, S.X64[nxt], sX, PC_DFS));
      RUN(OP64R(n2, S.X64[nxt], nxt));
    }
    RUN(set_act(g.act));
    RUN(DEFL(g.act, S.F[nxt] + 2L * m * L, sF, PC_C64));
    RUN(OP32(na, m, S.F[nxt] + 2L * m * L, sF, S.AF[nxt] + 2L * m * L, sF));
    g.cur = nxt;
    g.haveP = true;
    g.it = it + 1;
    return residual();
  }

 private:
  MixedShared &S;
  Group &g;
  pc_ctx *ctx;
};

}  // namespace

int solve_mixed(pc_ctx *ctx, int nb, const double *kr, std::vector<double> &gam, const std::vector<int> &zero,
                int nbands, int m, double tol, double *evals, void *evecs, int *iters, double *resid,
                std::vector<std::pair<int, int>> *handover) {
  const long n = ctx->n, L = 3 * n;
  const long sF = 3L * m * L, sX = (long)m * L;
  const int nmax = 3 * m;
  // default: 4 groups from 16 k-points (measured on the 40-k-point fcc batch: 60.1 k-points/s against 57.1 with 2
  // groups and 56.8 with 3), 2 from 8
  int ngroups = ctx->opts.groups > 0 ? ctx->opts.groups : (nb >= 16 ? 4 : (nb >= 8 ? 2 : 1));
  ngroups = std::max(1, std::min(ngroups, std::min(nb, pc_ctx::kMaxGroups)));
  PC_CK(ctx->S[0].reserve(sizeof(float2) * (size_t)sF * nb));
  PC_CK(ctx->S[1].reserve(sizeof(float2) * (size_t)sF * nb));
  PC_CK(ctx->AS[0].reserve(sizeof(float2) * (size_t)sF * nb));
  PC_CK(ctx->AS[1].reserve(sizeof(float2) * (size_t)sF * nb));
  PC_CK(ctx->X64[0].reserve(sizeof(float4) * (size_t)sX * nb));
  PC_CK(ctx->X64[1].reserve(sizeof(float4) * (size_t)sX * nb));
  PC_CK(ctx->R32.reserve(sizeof(float2) * (size_t)sX * nb));
  PC_CK(ctx->Gm.reserve(sizeof(double2) * (size_t)nb * nmax * nmax));
  PC_CK(ctx->Hm.reserve(sizeof(double2) * (size_t)nb * nmax * nmax));
  PC_CK(ctx->RQ.reserve(sizeof(double2) * (size_t)nb * m * nmax));
  PC_CK(ctx->GX.reserve(sizeof(double2) * (size_t)nb * m * m));
  PC_CK(ctx->coef.reserve(sizeof(double2) * (size_t)nb * nmax * m));
  PC_CK(ctx->theta.reserve(sizeof(double) * (size_t)nb * m));
  PC_CK(ctx->norms.reserve(sizeof(double) * (size_t)nb * m * 2));
  PC_CK(ctx->rnorm.reserve(sizeof(double) * (size_t)nb * m * 3));
  PC_CK(ctx->rank.reserve(sizeof(int) * (size_t)nb * (1 + ngroups)));
  PC_CK(ctx->flag.reserve(sizeof(int) * (size_t)nb));
  PC_CK(ctx->phase.reserve(sizeof(int) * (size_t)nb));
  PC_CK(ctx->mask.reserve(sizeof(int) * (size_t)nb * m));
  // scratch per group, sized for the group's largest k-point count
  const int gmax = (nb + ngroups - 1) / ngroups;
  // the chunked reductions' partial sums depend on the active count (not monotonically): size for every count
  size_t scr = 16;
  for (int na = 1; na <= gmax; ++na)
    scr = std::max({scr, gram_pair_scratch_bytes(na, L, nmax), gram_pair_coupled_scratch_bytes(na, L, nmax, m),
                    gram_df_scratch_bytes(na, L, m),
                    gram_scratch_bytes(na, L, m, nmax), residual_scratch_bytes(na, L, m),
                    recompute_scratch_bytes(n, na, m), op_df_resid_scratch_bytes(ctx, na, m),
                    deflate_scratch_bytes(na, m)});
  scr = (scr + 255) / 256 * 256;
  PC_CK(ctx->scratch.reserve(scr * ngroups));
  const size_t npin = (size_t)nb * m * 6;
  if (ctx->pinned_count < npin) {
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_count = 0;
    PC_CK(cudaMallocHost(&ctx->pinned, sizeof(double) * npin));
    ctx->pinned_count = npin;
  }
  for (int gi = 1; gi < ngroups; ++gi)
    if (!ctx->xstream[gi - 1]) PC_CK(cudaStreamCreateWithFlags(&ctx->xstream[gi - 1], cudaStreamNonBlocking));

  MixedShared S;
  S.ctx = ctx;
  S.nb = nb;
  S.nbands = nbands;
  S.m = m;
  S.n = n;
  S.L = L;
  S.sF = sF;
  S.sX = sX;
  S.nmax = nmax;
  S.tol = tol;
  // rank decision of the Rayleigh-Ritz (pivots of the unit-diagonal Gram): the complex64 products carry errors of
  // 1e-7 to 1e-6, so a direction whose independent part has a pivot near that is noise. Dropping below 1e-4 rather
  // than 1e-6 keeps such directions out of the pencil: on the diamond-air-N64 batch the mean iteration count fell
  // from 90.4 to 84.7 and the k-points whose phase 2 stalled or jumped from 6 to 1 (1e-5: 86.3 and 3).
  S.drop = 1e-4;
  S.kr = kr;
  S.gam = &gam;
  S.any_zero = false;
  for (int b = 0; b < nb; ++b) S.any_zero |= zero[b] != 0;
  S.zero = zero;
  for (int i = 0; i < 2; ++i) {
    S.F[i] = ctx->S[i].as<float2>();
    S.AF[i] = ctx->AS[i].as<float2>();
    S.X64[i] = ctx->X64[i].as<float4>();
  }
  S.R32 = ctx->R32.as<float2>();
  S.Gm = ctx->Gm.as<double2>();
  S.Hm = ctx->Hm.as<double2>();
  S.coef = ctx->coef.as<double2>();
  S.RQ = ctx->RQ.as<double2>();
  S.GX = ctx->GX.as<double2>();
  S.theta = ctx->theta.as<double>();
  S.norms = ctx->norms.as<double>();
  S.rn = ctx->rnorm.as<double>();
  S.d_zero = ctx->flag.as<int>();
  S.d_phase = ctx->phase.as<int>();
  S.d_mask = ctx->mask.as<int>();
  S.h_theta = ctx->pinned;
  S.h_norms = ctx->pinned + (size_t)nb * m;
  S.h_rn = ctx->pinned + (size_t)nb * m * 3;
  S.scr = scr;
  S.sG = (long)nmax * nmax;
  S.sRS = (long)m * nmax;
  S.sC = (long)nmax * m;
  S.phase.assign(nb, 1);
  S.doublings.assign(nb, 0);
  S.itcount.assign(nb, 0);
  S.done.assign(nb, 0);
  S.round_start.assign(nb, 0);
  S.p1_start.assign(nb, 0);
  S.hist.assign(nb, {});
  S.hist2.assign(nb, {});
  S.handover = handover;
  S.evals = evals;
  S.resid = resid;
  S.evecs = evecs;
  S.Ld = (double)L;
  S.nd = (double)n;
  S.fft_flops = 3.0 * 2.0 * 5.0 * S.nd * std::log2(S.nd) + 60.0 * S.nd;
  S.verbose = std::getenv("PC_VERBOSE") ? std::max(1, std::atoi(std::getenv("PC_VERBOSE"))) : 0;

  cudaStream_t st0 = ctx->stream;
  PC_CK(cudaMemcpyAsync(S.d_zero, zero.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st0));
  PC_CK(cudaMemcpyAsync(S.d_phase, S.phase.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st0));

  std::vector<Group> groups(ngroups);
  cudaEvent_t ready = nullptr;
  int rc = PC_OK;
  for (int gi = 0; gi < ngroups; ++gi) {
    Group &g = groups[gi];
    g.b0 = (int)((long)nb * gi / ngroups);
    g.b1 = (int)((long)nb * (gi + 1) / ngroups);
    g.st = gi == 0 ? st0 : ctx->xstream[gi - 1];
    g.d_act = ctx->rank.as<int>() + (size_t)nb * (1 + gi);
    g.scratch = static_cast<char *>(ctx->scratch.p) + scr * gi;
    PC_CK(cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming));
    PC_CK(cudaEventCreateWithFlags(&g.to_rr, cudaEventDisableTiming));
    PC_CK(cudaEventCreateWithFlags(&g.from_rr, cudaEventDisableTiming));
    if (!ctx->rrstream[gi]) {
      int lo = 0, hi = 0;
      PC_CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      PC_CK(cudaStreamCreateWithPriority(&ctx->rrstream[gi], cudaStreamNonBlocking, hi));
    }
    g.rst = ctx->rrstream[gi];
  }
  // the other groups' streams start after everything the caller's stream holds (setup, uploads above)
  if (ngroups > 1) {
    PC_CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    PC_CK(cudaEventRecord(ready, st0));
    for (int gi = 1; gi < ngroups; ++gi) PC_CK(cudaStreamWaitEvent(ctx->xstream[gi - 1], ready, 0));
  }
  for (int gi = 0; gi < ngroups && rc == PC_OK; ++gi) rc = MixedSolve(S, groups[gi]).start();
  // serve the groups in turn until all have finished
  while (rc == PC_OK) {
    bool any = false;
    for (int gi = 0; gi < ngroups && rc == PC_OK; ++gi) {
      Group &g = groups[gi];
      if (g.finished) continue;
      any = true;
      const cudaError_t e = cudaEventSynchronize(g.ev);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "cudaEventSynchronize(group)", __FILE__, __LINE__);
        break;
      }
      rc = harvest_timing(ctx);
      if (rc == PC_OK) rc = MixedSolve(S, g).step();
    }
    if (!any) break;
  }
  // join: the caller's stream waits for the other groups' work
  if (ngroups > 1) {
    for (int gi = 1; gi < ngroups; ++gi) {
      cudaEvent_t fin = nullptr;
      if (cudaEventCreateWithFlags(&fin, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(fin, ctx->xstream[gi - 1]);
        cudaStreamWaitEvent(st0, fin, 0);
        cudaEventDestroy(fin);
      }
    }
    cudaEventDestroy(ready);
  }
  const cudaError_t e0 = cudaStreamSynchronize(st0);
  for (auto &g : groups) {
    if (g.ev) cudaEventDestroy(g.ev);
    if (g.to_rr) cudaEventDestroy(g.to_rr);
    if (g.from_rr) cudaEventDestroy(g.from_rr);
  }
  if (rc != PC_OK) return rc;
  PC_CK(e0);
  PC_CK(cudaStreamSynchronize(st0));
  rc = harvest_timing(ctx);
  if (rc != PC_OK) return rc;
  if (iters)
    for (int b = 0; b < nb; ++b) iters[b] = S.itcount[b];
  return S.status;
}

#undef RUN

}  // namespace pc
