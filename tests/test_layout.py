"""The FP32 tile layout of the tensor-core contraction (tile_off in
csrc/prd_internal.h), checked on the host: the Re and Im halves each padded
to NP = N rounded up to 16 columns (ld = 2 NP); within a tile of N rows it is
injective from the 2N columns into [0, N ld), and every one of them lands in
the K step of its padded column (kp = k, or NP + k - N in the Im half), so no
K step mixes the halves; every K step is one contiguous block of N x 64 bytes
(one bulk copy, 16-byte aligned start and size); and inside a block each
row's 64 bytes are permuted by the 64-byte shared-memory swizzle, written here
in its own form (byte address bits [4:5] XOR bits [7:8]), which is the layout
the MMA descriptors declare.  The split layout of BF16x3 contexts
(tile_off_split: bf16 hi and lo planes in the same bytes) and the hi-only layout
of BF16x2 contexts (tile_off_hi: half the bytes) are checked the same way
against the 32-byte swizzle."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <cstdio>
#include <vector>
#include "prd_internal.h"
int main() {
  const int Ns[] = {1, 7, 8, 9, 150, 200, 208, 255, 256};
  for (int N : Ns) {
    const int NP = (N + 15) / 16 * 16, ld = 2 * NP;
    std::vector<char> seen((size_t)N * ld, 0);
    for (int n = 0; n < N; ++n)
      for (int k = 0; k < 2 * N; ++k) {
        const size_t off = prd::tile_off(n, k, N, ld, true);
        if (off >= (size_t)N * ld || seen[off]) { std::printf("N=%d n=%d k=%d: off %zu\n", N, n, k, off); return 1; }
        seen[off] = 1;
        const int kp = k < N ? k : NP + k - N;
        const int kc = kp / 16, kl = kp % 16;
        const size_t base = (size_t)kc * N * 16;            // floats
        if (off < base || off >= base + (size_t)N * 16) { std::printf("N=%d: step %d not contiguous\n", N, kc); return 2; }
        if ((kc < NP / 16) != (k < N)) { std::printf("N=%d k=%d: step mixes the halves\n", N, k); return 9; }
        const unsigned lin = (unsigned)(n * 64 + kl * 4);   // bytes, unswizzled row-major [n][16]
        const unsigned swz = lin ^ (((lin >> 7) & 3u) << 4);
        if ((off - base) * 4 != swz) { std::printf("N=%d n=%d k=%d: swizzle\n", N, n, k); return 3; }
        for (int lo = 0; lo < 2; ++lo) {
          const size_t o2 = prd::tile_off_split(n, k, N, ld, lo != 0);
          const size_t plane = (size_t)kc * N * 32 + (size_t)lo * N * 16;   // bf16 units
          if (o2 < plane || o2 >= plane + (size_t)N * 16) { std::printf("split N=%d: plane\n", N); return 7; }
          const unsigned l2 = (unsigned)(n * 32 + kl * 2);
          const unsigned s2 = l2 ^ (((l2 >> 7) & 1u) << 4);
          if ((o2 - plane) * 2 != s2) { std::printf("split N=%d n=%d k=%d: swizzle\n", N, n, k); return 8; }
        }
        // hi plane alone (BF16x2): chunk kc a block of N x 32 bytes, same swizzle
        const size_t oh = prd::tile_off_hi(n, k, N, ld);
        const size_t hp = (size_t)kc * N * 16;
        const unsigned l3 = (unsigned)(n * 32 + kl * 2);
        if (oh < hp || oh >= hp + (size_t)N * 16 || (oh - hp) * 2 != (l3 ^ (((l3 >> 7) & 1u) << 4))) {
          std::printf("hi N=%d n=%d k=%d\n", N, n, k);
          return 10;
        }
      }
    if (((size_t)N * ld * 4) % 64 || ((size_t)N * 64) % 16) { std::printf("N=%d: alignment\n", N); return 4; }
    if (prd::tile_off(N - 1, 2 * N - 1, N, 2 * N + 4, false) != (size_t)(N - 1) * (2 * N + 4) + 2 * N - 1) return 5;
  }
  std::printf("ok\n");
  return 0;
}
'''


def test_fp32_tile_layout_is_a_swizzled_bijection(tmp_path):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if not gxx or not os.path.isdir(cuda_inc):
        pytest.skip("g++ or the CUDA headers are missing")
    src = tmp_path / "layout.cpp"
    exe = tmp_path / "layout"
    src.write_text(SRC)
    csrc = os.path.join(ROOT, "paper_2505_20968_gb300", "csrc")
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-I", csrc, "-I", cuda_inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
