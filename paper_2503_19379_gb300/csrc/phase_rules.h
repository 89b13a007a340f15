// Host-side decisions of the mixed-precision solve on one k-point's residual history: when phase 1 (complex64
// block) gives way to phase 2 (FP64-accurate block), and when phase 2 hands the k-point to the FP64 finish.
// A history holds one entry per LOBPCG iteration, (iteration, largest relative residual of the wanted bands); a
// decision pass that repeats an iteration (phase switch, gamma doubling) does not add one. Plain C++ without CUDA,
// so that the rules are unit-tested on the host.
#pragma once
#include <algorithm>
#include <utility>
#include <vector>

namespace pc {

using ResidHistory = std::vector<std::pair<int, double>>;

// appends (it, mx) unless the last entry already is iteration it
inline void record_residual(ResidHistory &h, int it, double mx) {
  if (h.empty() || h.back().first != it) h.push_back({it, mx});
}

// the best of the last w entries is not below `factor` times the best of the w entries before them (false while the
// history holds fewer than 2w entries)
inline bool stalled_over(const ResidHistory &h, int w, double factor) {
  const int k = (int)h.size();
  if (w <= 0 || k < 2 * w) return false;
  double recent = 1e300, before = 1e300;
  for (int q = k - w; q < k; ++q) recent = std::min(recent, h[q].second);
  for (int q = k - 2 * w; q < k - w; ++q) before = std::min(before, h[q].second);
  return recent > factor * before;
}

// Phase 1 -> 2 once the complex64 residual stops falling. A short stall (5 iterations not 30% below the 5 before)
// counts below stall_level only: the plateaus higher up, near 1 while the search space builds up and near 0.2
// later, are not a floor. A long stall (10 not 30% below the 10 before) counts at any level: near Gamma the
// complex64 floor itself can lie above 1. Also below `floor`, or after `cap` iterations in phase 1.
struct Phase1Rule {
  double floor = 3e-3, stall_level = 0.05;
  int cap = 150;
};
inline bool phase1_done(const ResidHistory &h, double mx, int iters_in_phase, const Phase1Rule &r) {
  const int k = (int)h.size();
  const bool stalled =
      (k >= 10 && mx < r.stall_level && stalled_over(h, 5, 0.7)) || (k >= 20 && stalled_over(h, 10, 0.7));
  return stalled || mx < r.floor || iters_in_phase >= r.cap;
}

// Phase 2, for a k-point whose history (since its phase switch or restart) already holds iteration it:
//   converged when every wanted band is within the tolerance (ok);
//   rollback when the residual jumps to 1000 times its best of the earlier iterations, after that best was below
//     1e-2 (a Ritz pair of a nearly dependent direction taken into the block, which can blow it up): the block of
//     the previous iteration is handed to the FP64 finish;
//   handover when it stalls (largest residual below 1e-2, the best of its last 25 iterations not 20% below the
//     best of the 25 before, after at least 50) or reaches the iteration cap: its block is handed over;
//   continue otherwise.
enum class Phase2Step { kContinue, kConverged, kRollback, kHandover };
inline Phase2Step phase2_step(const ResidHistory &h, int it, bool ok, double mx, bool capped) {
  if (ok) return Phase2Step::kConverged;
  double best = 1e300;
  for (const auto &e : h)
    if (e.first != it) best = std::min(best, e.second);
  const int k = (int)h.size();
  if (k >= 3 && best < 1e-2 && mx > 1000.0 * best) return Phase2Step::kRollback;
  if ((k >= 50 && mx < 1e-2 && stalled_over(h, 25, 0.8)) || capped) return Phase2Step::kHandover;
  return Phase2Step::kContinue;
}

}  // namespace pc
