"""The library's initial-state draw (csrc/draw.cuh) obtains the FP32 rounding of the
FP64 expression u * 0.2 - 0.1 with one FP32 multiply and one fused multiply-add, and
rests that on an exhaustive comparison rather than an error bound. The header is plain C++,
so the host compiler checks it here against that FP64 expression for every one of
the 2^24 values the draw's 24-bit uniform takes, and checks its SplitMix64 stream
against the published first outputs for seed 0.

No GPU needed; the device compiles the same header, and the GPU parity tests compare
the device's draws with the oracle's.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_25762_gb300", "csrc")

HARNESS = r"""
#include <stdio.h>
#include <string.h>
#include "draw.cuh"
int main(void) {
  long bad = 0;
  for (uint32_t m = 0; m < (1u << 24); ++m) {
    double u = (double)m * (1.0 / 16777216.0);
    volatile double p = u * 0.2;   /* two FP64 roundings, no contraction */
    float want = (float)(p - 0.1);
    float got = qh::init_scale_u24(m);
    uint32_t wb, gb;
    memcpy(&wb, &want, 4);
    memcpy(&gb, &got, 4);
    if (wb != gb) {
      if (bad < 4) printf("mismatch m=%u want=%a got=%a\n", m, want, got);
      ++bad;
    }
  }
  /* SplitMix64 outputs 0..2 for initial state 0 (the generator's published values). */
  printf("%llu %llu %llu\n", (unsigned long long)qh::sm64_out(0, 0),
         (unsigned long long)qh::sm64_out(0, 1), (unsigned long long)qh::sm64_out(0, 2));
  printf("bad %ld\n", bad);
  return bad != 0;
}
"""


def test_integer_draw_equals_fp64_expression_for_every_uniform(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "draw_check.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "draw_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    lines = out.stdout.splitlines()
    assert out.returncode == 0 and lines[-1] == "bad 0", out.stdout
    assert [int(v) for v in lines[-2].split()] == [
        16294208416658607535, 7960286522194355700, 487617019471545679]
