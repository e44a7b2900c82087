"""The lockstep rounds of the batched solve (csrc/lockstep.h), on the host
with plain threads and a stand-in launcher: workers run a random number of
steps, with random work between them (a worker busy elsewhere, like one
forming its refinement residual, holds nobody up once the others wait), and
leave at random points.  Checked: no deadlock (a watchdog ends the run),
every arrival is served by exactly one round, a round holds each worker at
most once and only workers waiting in it, every worker sees its own round's
status, and the rounds are launched one at a time."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <atomic>
#include <chrono>
#include <cstdio>
#include <random>
#include <set>
#include <thread>
#include <vector>
#include "lockstep.h"
int main() {
  for (int trial = 0; trial < 40; ++trial) {
    const int n = 1 + trial % 13;
    prd::Lockstep<int> ls(n);
    std::atomic<int> in_launch{0}, bad{0};
    std::atomic<long long> served{0}, arrivals{0};
    std::vector<int> last_round(n, -1);
    int round_id = 0;
    auto launch = [&](const std::vector<int>& req) {
      if (in_launch.fetch_add(1) != 0) bad += 1;          // one round at a time
      std::set<int> seen(req.begin(), req.end());
      if (seen.size() != req.size()) bad += 1;            // each worker once
      for (int w : req) last_round[w] = round_id;
      served += (long long)req.size();
      const int status = 1000 + round_id++;
      in_launch.fetch_sub(1);
      return status;
    };
    std::vector<std::thread> th;
    for (int w = 0; w < n; ++w)
      th.emplace_back([&, w]() {
        std::mt19937 rng(1234 + 97 * trial + w);
        const int steps = rng() % 25;
        for (int k = 0; k < steps; ++k) {
          if (rng() % 3 == 0) std::this_thread::sleep_for(std::chrono::microseconds(rng() % 200));
          arrivals += 1;
          const int st = ls.arrive(w, launch);
          if (st != 1000 + last_round[w]) bad += 1;       // the status of its own round
        }
        ls.leave(launch);
      });
    for (auto& t : th) t.join();
    if (bad || served != arrivals) {
      std::printf("trial %d: bad %d served %lld arrivals %lld\n", trial, bad.load(), served.load(), arrivals.load());
      return 1;
    }
  }
  std::printf("ok\n");
  return 0;
}
'''


def test_lockstep_rounds_serve_every_arrival_once(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ is missing")
    src = tmp_path / "lockstep.cpp"
    exe = tmp_path / "lockstep"
    src.write_text(SRC)
    csrc = os.path.join(ROOT, "paper_2505_20968_gb300", "csrc")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-pthread", "-I", csrc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)   # the deadlock watchdog
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
