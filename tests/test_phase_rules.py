"""The mixed solve's host-side decisions (paper_2503_19379_gb300/csrc/phase_rules.h) on synthetic residual
histories: when phase 1 (complex64 block) switches to phase 2 (FP64-accurate block), and when phase 2 hands a
k-point to the FP64 finish (a stall, a jump, the iteration cap). The header is plain C++; the test compiles a small
driver with g++ and checks the iteration at which each rule fires."""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2503_19379_gb300", "csrc")

DRIVER = r"""
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>
#include "phase_rules.h"
using namespace pc;

// first iteration at which phase 1 would switch for the residual sequence r (-1: never)
static int phase1_first(const std::vector<double> &r) {
  ResidHistory h;
  for (int it = 0; it < (int)r.size(); ++it) {
    record_residual(h, it, r[it]);
    if (phase1_done(h, r[it], it, Phase1Rule{})) return it;
  }
  return -1;
}
// first phase-2 decision other than kContinue: (iteration, code 1 converged / 2 rollback / 3 handover), or (-1, 0)
static std::pair<int, int> phase2_first(const std::vector<double> &r, double tol, int maxiter) {
  ResidHistory h;
  for (int it = 0; it < (int)r.size(); ++it) {
    record_residual(h, it, r[it]);
    const Phase2Step s = phase2_step(h, it, r[it] <= tol, r[it], it >= maxiter);
    if (s != Phase2Step::kContinue) return {it, (int)s};
  }
  return {-1, 0};
}
static void emit(const char *name, int a, int b = 0) { std::printf("\"%s\": [%d, %d],\n", name, a, b); }

int main() {
  std::printf("{\n");
  // phase 1: steady convergence 0.8^k from 1: switches when it passes the 3e-3 floor
  std::vector<double> geo;
  for (int k = 0; k < 200; ++k) geo.push_back(std::pow(0.8, k));
  emit("p1_geometric", phase1_first(geo));
  // phase 1: a plateau at 0.2 from iteration 5 on: only the long-stall rule (10 vs 10) applies above 0.05
  std::vector<double> hi(200, 0.2);
  for (int k = 0; k < 5; ++k) hi[k] = 1.0 + k;
  emit("p1_plateau_0.2", phase1_first(hi));
  // phase 1: a plateau at 0.02 from iteration 5 on: the short-stall rule (5 vs 5) applies below 0.05
  std::vector<double> lo(200, 0.02);
  for (int k = 0; k < 5; ++k) lo[k] = 1.0 + k;
  emit("p1_plateau_0.02", phase1_first(lo));
  // phase 1: steady progress of 0.962 per iteration (32% per 10) from 50, above 0.05 for 150 iterations: no
  // stall, the 150-iteration cap decides; at 0.97 per iteration (26% per 10) the long-stall rule fires instead
  std::vector<double> slow, slower;
  for (int k = 0; k < 200; ++k) slow.push_back(50.0 * std::pow(0.962, k));
  for (int k = 0; k < 200; ++k) slower.push_back(50.0 * std::pow(0.97, k));
  emit("p1_slow", phase1_first(slow));
  emit("p1_slower", phase1_first(slower));
  // a repeated decision pass (same iteration recorded twice) adds one entry
  {
    ResidHistory h;
    record_residual(h, 3, 0.5);
    record_residual(h, 3, 0.4);
    record_residual(h, 4, 0.3);
    emit("record_entries", (int)h.size(), (int)(h[0].second * 10 + 0.5));
  }
  // phase 2: 0.8 per iteration from 0.5 converges to 1e-6 with no other decision
  std::vector<double> conv;
  for (int k = 0; k < 200; ++k) conv.push_back(0.5 * std::pow(0.8, k));
  auto c = phase2_first(conv, 1e-6, 400);
  emit("p2_converges", c.first, c.second);
  // phase 2: fast to 3e-6 by iteration 40, then bouncing between 3e-6 and 7e-6: handed over once 25 iterations
  // bring no 20% gain over the 25 before (and at least 50 entries)
  std::vector<double> plat;
  for (int k = 0; k < 200; ++k) plat.push_back(k < 40 ? 0.5 * std::pow(0.74, k) : (k % 3 == 0 ? 7e-6 : 3e-6));
  auto p = phase2_first(plat, 1e-6, 400);
  emit("p2_plateau", p.first, p.second);
  // phase 2: a jump of 2000x after reaching 1e-5 is rolled back; one of 100x is not
  std::vector<double> jump;
  for (int k = 0; k < 60; ++k) jump.push_back(k < 30 ? 0.5 * std::pow(0.7, k) : 1e-5);
  const double best = jump[29];
  jump[45] = 100.0 * best;
  jump[50] = 2000.0 * best;
  auto j = phase2_first(jump, 1e-12, 400);
  emit("p2_jump", j.first, j.second);
  // phase 2: the iteration cap hands over
  std::vector<double> capv;
  for (int k = 0; k < 30; ++k) capv.push_back(0.5 * std::pow(0.95, k));
  auto cp = phase2_first(capv, 1e-6, 20);
  emit("p2_cap", cp.first, cp.second);
  // phase 2: a residual still above 1e-2 is never handed over for a stall
  std::vector<double> high(120, 0.05);
  auto hh = phase2_first(high, 1e-6, 400);
  emit("p2_high_plateau", hh.first, hh.second);
  std::printf("\"end\": [0, 0]\n}\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("phase_rules")
    src, exe = d / "driver.cpp", d / "driver"
    src.write_text(DRIVER)
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def test_phase1_switches_at_the_floor_on_steady_convergence(results):
    # 0.8^k < 3e-3 first at k = 27 (0.8^26 = 3.02e-3)
    assert results["p1_geometric"][0] == 27


def test_phase1_long_stall_fires_at_any_level(results):
    # 20 entries are needed for the 10-vs-10 window; entries 0..19, the window's halves both at 0.2 from entry 5
    assert results["p1_plateau_0.2"][0] == 19


def test_phase1_short_stall_fires_below_its_level(results):
    # entries 0..4 lie above 1, so at entry 9 the last 5 (0.02) are far below the 5 before (best 1); at entry 10
    # the earlier window (1..5) already holds the first 0.02 (entry 5), so the last 5 (6..10) are not 30% below it:
    # the 5-vs-5 rule fires there, long before the 10-vs-10 rule could (entry 19)
    assert results["p1_plateau_0.02"][0] == 10


def test_phase1_cap(results):
    # 0.962^10 = 0.68 < 0.7: never a stall, and 50 * 0.962^150 = 0.15 stays above both 0.05 and the floor
    assert results["p1_slow"][0] == 150
    # 0.97^10 = 0.74 > 0.7: the 10-vs-10 rule fires as soon as it has 20 entries
    assert results["p1_slower"][0] == 19


def test_a_repeated_pass_keeps_one_entry(results):
    assert results["record_entries"] == [2, 5]


def test_phase2_converges_without_handover(results):
    it, code = results["p2_converges"]
    assert code == 1 and 0.5 * 0.8 ** it <= 1e-6 < 0.5 * 0.8 ** (it - 1)


def test_phase2_plateau_is_handed_over(results):
    it, code = results["p2_plateau"]
    assert code == 3
    # the plateau (best value 3e-6) starts at entry 40 (0.5 * 0.74^39 = 4e-6 just before it). The stall shows when
    # the earlier window first reaches the plateau: at entry 65 the windows are 16..40 and 41..65, both with best
    # 3e-6, so the last 25 are not 20% below the 25 before
    assert it == 65


def test_phase2_jump_is_rolled_back(results):
    it, code = results["p2_jump"]
    assert (it, code) == (50, 2)  # the 100x excursion at 45 passes; the 2000x one at 50 rolls back


def test_phase2_cap_hands_over(results):
    assert results["p2_cap"] == [20, 3]


def test_phase2_no_stall_handover_above_1e_2(results):
    assert results["p2_high_plateau"] == [-1, 0]
