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
// * The X-X block (X^H X, X^H AX) and the residual need FP64: the residual floor of a complex64 X is eps32 |Op| / lambda
//   (about 1e-3 here), and the X-X block's rounding shifts the Ritz values by eps32 lambda.
// Phase 1 (every k-point starts here): X and AX in complex64 as well, until the complex64 residual stops falling.
// Phase 2: X, AX stored in FP64; X' = X C_X + P' (complex64 correction), AX' by the stencil and the X-X block, all
// three in double-float arithmetic (mixed_df.cu) on the FP32 pipe.
// Convergence and Algorithm 4.1 are decided in phase 2 only, on FP64 residuals and FP64 norms.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pc_internal.cuh"

namespace pc {

int solve_mixed(pc_ctx *ctx, int nb, const double *kr, std::vector<double> &gam, const std::vector<int> &zero,
                int nbands, int m, double tol, double *evals, void *evecs, int *iters, double *resid) {
  cudaStream_t st = ctx->stream;
  const long n = ctx->n, L = 3 * n;
  const long sF = 3L * m * L, sX = (long)m * L;
  const int nmax = 3 * m;
  PC_CK(ctx->S[0].reserve(sizeof(float2) * (size_t)sF * nb));
  PC_CK(ctx->S[1].reserve(sizeof(float2) * (size_t)sF * nb));
  PC_CK(ctx->AS[0].reserve(sizeof(float2) * (size_t)sF * nb));
  PC_CK(ctx->AS[1].reserve(sizeof(float2) * (size_t)sF * nb));
  PC_CK(ctx->X64[0].reserve(sizeof(double2) * (size_t)sX * nb));
  PC_CK(ctx->X64[1].reserve(sizeof(double2) * (size_t)sX * nb));
  PC_CK(ctx->AX64.reserve(sizeof(double2) * (size_t)sX * nb));
  PC_CK(ctx->R32.reserve(sizeof(float2) * (size_t)sX * nb));
  PC_CK(ctx->Gm.reserve(sizeof(double2) * (size_t)nb * nmax * nmax));
  PC_CK(ctx->Hm.reserve(sizeof(double2) * (size_t)nb * nmax * nmax));
  PC_CK(ctx->RQ.reserve(sizeof(double2) * (size_t)nb * m * 2 * m));
  PC_CK(ctx->GX.reserve(sizeof(double2) * (size_t)nb * m * m));
  PC_CK(ctx->HX.reserve(sizeof(double2) * (size_t)nb * m * m));
  PC_CK(ctx->coef.reserve(sizeof(double2) * (size_t)nb * nmax * m));
  PC_CK(ctx->theta.reserve(sizeof(double) * (size_t)nb * m));
  PC_CK(ctx->norms.reserve(sizeof(double) * (size_t)nb * m * 2));
  PC_CK(ctx->rnorm.reserve(sizeof(double) * (size_t)nb * m * 3));
  PC_CK(ctx->rank.reserve(sizeof(int) * (size_t)nb * 2));
  PC_CK(ctx->flag.reserve(sizeof(int) * (size_t)nb));
  PC_CK(ctx->phase.reserve(sizeof(int) * (size_t)nb));
  const size_t scr = std::max({gram_pair_scratch_bytes(nb, L, nmax), gram_df_scratch_bytes(nb, L, m),
                               gram_scratch_bytes(nb, L, m, 2 * m), residual_scratch_bytes(nb, L, m),
                               sizeof(double2) * (size_t)nb * 3 * m * 16, sizeof(double) * 3 * (size_t)nb * m * 64,
                               (size_t)16});
  PC_CK(ctx->scratch.reserve(scr));
  void *scratch = ctx->scratch.p;
  float2 *F[2] = {ctx->S[0].as<float2>(), ctx->S[1].as<float2>()};
  float2 *AF[2] = {ctx->AS[0].as<float2>(), ctx->AS[1].as<float2>()};
  double2 *X64[2] = {ctx->X64[0].as<double2>(), ctx->X64[1].as<double2>()};
  double2 *AX64 = ctx->AX64.as<double2>();
  float2 *R32 = ctx->R32.as<float2>();
  double2 *Gm = ctx->Gm.as<double2>(), *Hm = ctx->Hm.as<double2>(), *coef = ctx->coef.as<double2>();
  double2 *RQ = ctx->RQ.as<double2>(), *GX = ctx->GX.as<double2>(), *HX = ctx->HX.as<double2>();
  double *theta = ctx->theta.as<double>(), *norms = ctx->norms.as<double>(), *rn = ctx->rnorm.as<double>();
  int *d_act = ctx->rank.as<int>() + nb;
  int *d_zero = ctx->flag.as<int>();
  int *d_phase = ctx->phase.as<int>();
  PC_CK(ctx->mask.reserve(sizeof(int) * (size_t)nb * m));
  int *d_mask = ctx->mask.as<int>();
  uint64_t restarts = 0;
  const double drop = 1e-12;

  std::vector<int> phase(nb, 1), doublings(nb, 0), itcount(nb, 0), done(nb, 0), round_start(nb, 0), p1_start(nb, 0);
  std::vector<std::vector<double>> hist(nb);
  PC_CK(cudaMemcpyAsync(d_zero, zero.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
  PC_CK(cudaMemcpyAsync(d_phase, phase.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
  bool any_zero = false;
  for (int b = 0; b < nb; ++b) any_zero |= zero[b] != 0;

  // algorithmic work per stage invocation: 8 bytes per complex64 entry, 16 per FP64 entry
  const double Ld = (double)L, nd = (double)n;
  const double fft_flops = 3.0 * 2.0 * 5.0 * nd * std::log2(nd) + 60.0 * nd;
  auto set_act = [&](const std::vector<int> &v) -> int {
    if (v.empty()) return PC_OK;
    PC_CK(cudaMemcpyAsync(d_act, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, st));
    return PC_OK;
  };
  auto OP32 = [&](int nbk, int cols, const void *X, long sx, void *Y, long sy) {
    return run_stage(ctx, PC_STAGE_STENCIL, 1, 214.0 * nd * nbk * cols, 2.0 * Ld * 8.0 * nbk * cols + 12.0 * nd,
                     [&] { return launch_apply_op(ctx, nbk, cols, PC_C64, X, sx, Y, sy, d_act); });
  };
  auto OP64 = [&](int nbk, const void *X, void *Y) {  // FP64 block, double-float arithmetic
    return run_stage(ctx, PC_STAGE_STENCIL, 1, 214.0 * nd * nbk * m, 2.0 * Ld * 16.0 * nbk * m + 24.0 * nd,
                     [&] { return launch_apply_op_df(ctx, nbk, m, X, sX, Y, sX, d_act); });
  };
  auto DEFL = [&](int nbk, void *X, long sx, int dtype) {
    return run_stage(ctx, PC_STAGE_OTHER, 2, 4.0 * Ld * m * nbk, 2.0 * Ld * (dtype == PC_C64 ? 8.0 : 16.0) * m * nbk,
                     [&] { return launch_deflate(nbk, n, m, X, sx, d_zero, scratch, st, d_act, dtype); });
  };
#define RUN(x)                    \
  do {                            \
    int rc_ = (x);                \
    if (rc_ != PC_OK) return rc_; \
  } while (0)

  std::vector<int> act;
  for (int b = 0; b < nb; ++b) act.push_back(b);
  RUN(set_act(act));
  // ---- initial block (FP64 generator, narrowed) and Rayleigh-Ritz on span(X0), all in phase 1
  RUN(run_stage(ctx, PC_STAGE_OTHER, 1, 0.0, Ld * 16.0 * m * nb,
                [&] { return launch_init_block(nb, L, m, ctx->opts.seed, 0, X64[0], sX, st); }));
  if (any_zero) RUN(DEFL(nb, X64[0], sX, PC_C128));
  RUN(run_stage(ctx, PC_STAGE_OTHER, 1, 0.0, Ld * 24.0 * m * nb,
                [&] { return launch_narrow(nb, L, m, X64[0], sX, F[0], sF, st, d_act); }));
  RUN(OP32(nb, m, F[0], sF, AF[0], sF));
  RUN(run_stage(ctx, PC_STAGE_GRAM, 2, 8.0 * m * (m + 1) * Ld * nb, 2.0 * m * Ld * 8.0 * nb, [&] {
    return launch_gram_pair(nb, L, m, PC_C64, F[0], AF[0], sF, Gm, Hm, scratch, scr, st, d_act, nb);
  }));
  RUN(run_stage(ctx, PC_STAGE_RR, 1, 0.0, 2.0 * m * m * 16.0 * nb,
                [&] { return launch_rr(nb, m, m, Gm, Hm, drop, theta, coef, nullptr, st, d_act); }));
  RUN(run_stage(ctx, PC_STAGE_UPDATE, 1, 8.0 * m * m * Ld * nb, 2.0 * m * Ld * 8.0 * nb, [&] {
    return launch_block_update(nb, L, m, m, PC_C64, F[0], sF, coef, (long)m * m, F[1], sF, st, d_act);
  }));
  RUN(OP32(nb, m, F[1], sF, AF[1], sF));
  int cur = 1;
  bool haveP = false;

  std::vector<double> h_theta((size_t)nb * m), h_norms((size_t)nb * m * 2), h_rn((size_t)nb * m * 3);
  int status = PC_OK;
  const int maxiter = ctx->opts.maxiter;
  for (int it = 0;; ++it) {
    std::vector<int> act1, act2;
    for (int b : act) (phase[b] == 1 ? act1 : act2).push_back(b);
    const int nxt = 1 - cur;
    // ---- residuals: complex64 block (phase 1) or FP64 block with complex64 copies of X, AX (phase 2)
    if (!act1.empty()) {
      RUN(set_act(act1));
      const int na = (int)act1.size();
      RUN(run_stage(ctx, PC_STAGE_RESIDUAL, 2, 8.0 * Ld * m * na, 4.0 * Ld * 8.0 * m * na, [&] {
        return launch_residual_mixed(na, L, m, PC_C64, F[cur], sF, AF[cur], sF, theta, F[cur] + (long)m * L, sF,
                                     R32, sX, nullptr, 0, nullptr, 0, norms, scratch, scr, st, d_act);
      }));
    }
    if (!act2.empty()) {
      RUN(set_act(act2));
      const int na = (int)act2.size();
      RUN(run_stage(ctx, PC_STAGE_RESIDUAL, 2, 8.0 * Ld * m * na, (2.0 * 16.0 + 4.0 * 8.0) * Ld * m * na, [&] {
        return launch_residual_mixed(na, L, m, PC_C128, X64[cur], sX, AX64, sX, theta, F[cur] + (long)m * L, sF, R32,
                                     sX, F[cur], sF, AF[cur], sF, norms, scratch, scr, st, d_act);
      }));
    }
    PC_CK(cudaMemcpyAsync(h_theta.data(), theta, sizeof(double) * nb * m, cudaMemcpyDeviceToHost, st));
    PC_CK(cudaMemcpyAsync(h_norms.data(), norms, sizeof(double) * nb * m * 2, cudaMemcpyDeviceToHost, st));
    PC_CK(cudaStreamSynchronize(st));
    RUN(harvest_timing(ctx));
    auto relres = [&](int b, int j) {
      const double r = h_norms[((size_t)b * m + j) * 2], x = h_norms[((size_t)b * m + j) * 2 + 1];
      return r / (std::fabs(h_theta[(size_t)b * m + j]) * x);
    };
    // ---- phase 1 -> 2 when the complex64 residual stops falling (or is already small)
    std::vector<int> sw;
    for (int b : act1) {
      double mx = 0;
      for (int j = 0; j < nbands; ++j) mx = std::max(mx, relres(b, j));
      if (!(mx == mx)) mx = 1e300;  // NaN guard
      hist[b].push_back(mx);
      const int k1 = (int)hist[b].size();
      const bool stalled = k1 > 8 && mx > 0.7 * hist[b][k1 - 6];
      if (stalled || mx < 1e-4 || it - p1_start[b] >= 150) sw.push_back(b);
    }
    // ---- phase 2: convergence on FP64 residuals, then Algorithm 4.1
    std::vector<int> conv;
    for (int b : act2) {
      bool ok = true;
      for (int j = 0; j < nbands; ++j)
        if (!(relres(b, j) <= tol)) ok = false;
      if (ok || it - round_start[b] >= maxiter) conv.push_back(b);
    }
    std::vector<int> redo, fin;
    if (!conv.empty()) {
      RUN(set_act(conv));
      const int nc = (int)conv.size();
      RUN(run_stage(ctx, PC_STAGE_RECOMPUTE, 2, 120.0 * nd * m * nc, Ld * 16.0 * m * nc,
                    [&] { return launch_recompute(ctx, nc, m, X64[cur], sX, rn, d_act); }));
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
        if (resid) resid[(size_t)b * nbands + j] = relres(b, j);
      }
      if (evecs)
        PC_CK(cudaMemcpyAsync(static_cast<double2 *>(evecs) + (size_t)b * nbands * L, X64[cur] + (size_t)b * sX,
                              sizeof(double2) * (size_t)nbands * L, cudaMemcpyDeviceToDevice, st));
    }
    {
      std::vector<int> keep;
      for (int b : act)
        if (!done[b]) keep.push_back(b);
      act.swap(keep);
    }
    if (act.empty()) break;
    if (!sw.empty() || !redo.empty()) {
      // phase switch: X64 = X (widened), AX64 = Op X64; gamma doubling: AX64 and AP with the new gamma
      if (!sw.empty()) {
        for (int b : sw) {
          phase[b] = 2;
          round_start[b] = it + 1;
        }
        RUN(set_act(sw));
        const int ns = (int)sw.size();
        RUN(run_stage(ctx, PC_STAGE_OTHER, 1, 0.0, Ld * 24.0 * m * ns,
                      [&] { return launch_widen(ns, L, m, F[cur], sF, X64[cur], sX, st, d_act); }));
        RUN(OP64(ns, X64[cur], AX64));
        PC_CK(cudaMemcpyAsync(d_phase, phase.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
      }
      if (!redo.empty()) {
        for (int b : redo) {
          gam[b] *= 2.0;
          doublings[b] += 1;
          round_start[b] = it + 1;
        }
        RUN(upload_kpoints(ctx, nb, kr, gam.data()));
        RUN(set_act(redo));
        const int nr = (int)redo.size();
        // spurious columns (gamma-independent exact eigenvectors of B'B) are replaced by fresh random columns
        std::vector<int> mask((size_t)nb * m);
        spurious_mask(redo, m, nbands, tol, h_theta, h_rn, mask);
        PC_CK(cudaMemcpyAsync(d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, st));
        ++restarts;
        RUN(run_stage(ctx, PC_STAGE_OTHER, 1, 0.0, 0.0, [&] {
          return launch_init_block(nr, L, m, ctx->opts.seed + 7919ULL * restarts, 0, X64[cur], sX, st, d_mask, d_act);
        }));
        if (any_zero) RUN(DEFL(nr, X64[cur], sX, PC_C128));
        RUN(OP64(nr, X64[cur], AX64));
        if (haveP) RUN(OP32(nr, m, F[cur] + 2L * m * L, sF, AF[cur] + 2L * m * L, sF));
      }
      continue;  // residuals again with the new block or operator
    }
    const int nc = haveP ? 3 * m : 2 * m;
    const int nq = nc - m;
    act1.clear();
    act2.clear();
    for (int b : act) (phase[b] == 1 ? act1 : act2).push_back(b);
    RUN(set_act(act));
    const int na = (int)act.size();
    // ---- W = P^{-1} R (complex64), AW = Op W
    RUN(run_stage(ctx, PC_STAGE_PRECOND, 5, fft_flops * na * m, 2.0 * Ld * 8.0 * na * m, [&] {
      return launch_precond(ctx, na, m, PC_C64, F[cur] + (long)m * L, sF, F[cur] + (long)m * L, sF, d_act);
    }));
    if (any_zero) RUN(DEFL(na, F[cur] + (long)m * L, sF, PC_C64));
    RUN(OP32(na, m, F[cur] + (long)m * L, sF, AF[cur] + (long)m * L, sF));
    // ---- pencil: complex64 products over [X | W | P], the R^H Q coupling, FP64 X-X block in phase 2
    RUN(run_stage(ctx, PC_STAGE_GRAM, 2, 8.0 * nc * (nc + 1) * Ld * na, 2.0 * nc * Ld * 8.0 * na, [&] {
      return launch_gram_pair(na, L, nc, PC_C64, F[cur], AF[cur], sF, Gm, Hm, scratch, scr, st, d_act, nb);
    }));
    RUN(run_stage(ctx, PC_STAGE_GRAM, 2, 8.0 * m * nq * Ld * na, (double)(m + nq) * Ld * 8.0 * na, [&] {
      return launch_gram(na, L, m, nq, PC_C64, R32, sX, F[cur] + (long)m * L, sF, RQ, scratch, scr, st, d_act,
                         nb);
    }));
    if (!act2.empty()) {
      RUN(set_act(act2));
      const int n2 = (int)act2.size();
      RUN(run_stage(ctx, PC_STAGE_GRAM, 2, 8.0 * m * (m + 1) * Ld * n2, 2.0 * m * Ld * 16.0 * n2, [&] {
        return launch_gram_df(n2, L, m, X64[cur], AX64, sX, GX, HX, scratch, scr, st, d_act);
      }));
      RUN(set_act(act));
    }
    RUN(run_stage(ctx, PC_STAGE_RR, 1, 0.0, 2.0 * nc * nc * 16.0 * na, [&] {
      int rc = launch_rr_patch(na, nc, m, Gm, Hm, RQ, theta, GX, HX, d_phase, st, d_act);
      if (rc) return rc;
      return launch_rr(na, nc, m, Gm, Hm, drop, theta, coef, nullptr, st, d_act);
    }));
    // ---- P' = [W P] coef_{W,P} (complex64), then X' per phase
    RUN(run_stage(ctx, PC_STAGE_UPDATE, 1, 8.0 * nq * m * Ld * na, (double)(nq + m) * Ld * 8.0 * na, [&] {
      return launch_block_update(na, L, nq, m, PC_C64, F[cur] + (long)m * L, sF, coef + (long)m * m, (long)nc * m,
                                 F[nxt] + 2L * m * L, sF, st, d_act);
    }));
    if (!act1.empty()) {
      RUN(set_act(act1));
      const int n1 = (int)act1.size();
      RUN(run_stage(ctx, PC_STAGE_UPDATE, 1, 8.0 * nc * m * Ld * n1, (double)(nc + m) * Ld * 8.0 * n1, [&] {
        return launch_block_update(n1, L, nc, m, PC_C64, F[cur], sF, coef, (long)nc * m, F[nxt], sF, st, d_act);
      }));
      if (any_zero) RUN(DEFL(n1, F[nxt], sF, PC_C64));
      RUN(OP32(n1, m, F[nxt], sF, AF[nxt], sF));
    }
    if (!act2.empty()) {
      RUN(set_act(act2));
      const int n2 = (int)act2.size();
      RUN(run_stage(ctx, PC_STAGE_UPDATE, 1, 8.0 * m * m * Ld * n2, (2.0 * 16.0 + 8.0) * m * Ld * n2, [&] {
        return launch_update_df(n2, L, m, m, X64[cur], sX, coef, (long)nc * m, X64[nxt], sX, F[nxt] + 2L * m * L,
                                sF, st, d_act);
      }));
      if (any_zero) RUN(DEFL(n2, X64[nxt], sX, PC_C128));
      RUN(OP64(n2, X64[nxt], AX64));
    }
    RUN(set_act(act));
    if (any_zero) RUN(DEFL(na, F[nxt] + 2L * m * L, sF, PC_C64));
    RUN(OP32(na, m, F[nxt] + 2L * m * L, sF, AF[nxt] + 2L * m * L, sF));
    cur = nxt;
    haveP = true;
  }
#undef RUN
  PC_CK(cudaStreamSynchronize(st));
  if (iters)
    for (int b = 0; b < nb; ++b) iters[b] = itcount[b];
  return status;
}

}  // namespace pc
