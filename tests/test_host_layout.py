"""CPU test of the host-memory solve's workspace layout
(paper_2107_05395_gb300/csrc/host_layout.h, compiled here on its own).

Every slot of the workspace holds one chunk's right-hand sides and then its
solutions.  With FP32 right-hand sides and FP64 solutions an odd N * chunk would put
the solution part 4 bytes off an 8-byte boundary if the parts were packed, so both
parts (and hence every slot) must start on a 256-byte boundary and still hold all
of their elements without overlapping."""
import ctypes
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("hostlayout") / "host_layout.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-o", out,
                    os.path.join(HERE, "native", "host_layout_harness.cpp")], check=True)
    L = ctypes.CDLL(out)
    L.h_slot_x_offset.restype = ctypes.c_ulong
    L.h_slot_x_offset.argtypes = [ctypes.c_long, ctypes.c_long, ctypes.c_ulong]
    L.h_slot_bytes.restype = ctypes.c_ulong
    L.h_slot_bytes.argtypes = [ctypes.c_long, ctypes.c_long, ctypes.c_ulong, ctypes.c_ulong]
    return L


@pytest.mark.parametrize("N", [1, 5, 7, 255, 1023])
@pytest.mark.parametrize("C", [1, 3, 17, 4097])
@pytest.mark.parametrize("rs,xs", [(4, 8), (8, 4), (4, 4), (8, 8)])
def test_every_part_of_every_slot_is_aligned_and_disjoint(H, N, C, rs, xs):
    x_off = H.h_slot_x_offset(N, C, rs)
    slot = H.h_slot_bytes(N, C, rs, xs)
    assert x_off >= N * C * rs, "the right-hand sides overrun the solution part"
    assert slot - x_off >= N * C * xs, "the solutions overrun the slot"
    assert x_off - N * C * rs < 256 and slot - x_off - N * C * xs < 256, "padding beyond one boundary"
    for k in range(H.h_slots()):
        assert (k * slot) % 256 == 0 and (k * slot + x_off) % 256 == 0
