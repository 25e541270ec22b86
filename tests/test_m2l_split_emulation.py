"""Host emulation of the mixed-precision M2L (Sec. 2.3 translations,
tests/emu/m2l_split_emu.cpp): the far field of one observer box's 189
interaction-list sources, M2L'd with FP64, 3xTF32 and three-product FP16
splits, then L2P'd.  It pins the design of the tensor-core M2L's operands:
with the power-of-two scales (level inputs into (2^14, 2^15], operator
columns into (2^13, 2^14]) the FP16 split is as accurate as 3xTF32 even with
FP16 subnormals flushed, while unit scales lose three orders of magnitude.
The GPU kernel itself is checked against the oracle by the GPU tests."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("emu") / "m2l_split_emu")
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1107_5951_gb300", "csrc"),
                        "-o", exe, os.path.join(ROOT, "tests", "emu", "m2l_split_emu.cpp")],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("emulation does not build here (needs _Float16): " + r.stderr[-300:])
    return exe


@pytest.mark.parametrize("p,mode", [(8, 2), (12, 0), (12, 1)])
def test_fp16_split_with_scales_matches_3xtf32(emu, p, mode):
    out = subprocess.run([emu, str(p), str(mode)], capture_output=True, text=True, check=True).stdout
    trunc, tf32, f16, f16_unit = (float(x) for x in out.split())
    # the harness itself: the FP64 M2L + L2P reproduces the direct sum to the
    # truncation error of the expansion (positive densities, p = 12)
    if mode == 0 and p == 12:
        assert trunc < 1e-5
    assert f16 <= 2.0 * tf32 + 1e-7
    assert f16 <= 1e-6
    assert f16_unit >= 100.0 * f16
