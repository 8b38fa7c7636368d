"""Host-side checks of the tcgen05 GEMM's shared-memory layout and
descriptors (`umma.cuh`; no GPU: a small host program compiled with nvcc
evaluates the constexpr encoders).  Field positions follow the PTX ISA's
tcgen05 shared-memory matrix descriptor (start address >> 4 in bits 0-13,
leading byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45,
version 1 in 46-47, base offset in 49-51, leading-offset mode in 52, layout
type in 61-63; 128-byte swizzle = 2) and instruction descriptor of
kind::f16 (D format in 4-5, A and B formats in 7-9 and 10-12, negations in
13-14, A and B major in 15-16, N >> 3 in 17-22, M >> 4 in 24-28)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_02134_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "umma.cuh"
using namespace sem;
int main() {
  for (int r = 0; r < kUM; ++r)
    for (int c = 0; c < kUK / 8; ++c) std::printf("off %d %d %u\n", r, c, umma_chunk_off(r, c));
  const unsigned addrs[] = {0u, 1024u, 16384u + 32u, 65536u + 96u, 131072u};
  for (unsigned a : addrs)
    std::printf("desc %u %llu\n", a, (unsigned long long)umma_desc(a));
  std::printf("idesc %u\n", umma_idesc(kUM, kUN));
  std::printf("smem %zu %d %u %u %d\n", kUSmem, kUStages, kUTileA, kUTileB, (int)kUCols);
  return 0;
}
"""


@pytest.fixture(scope="module")
def values():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "umma_layout.cu")
        exe = os.path.join(d, "umma_layout")
        open(src, "w").write(PROGRAM)
        r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                            "-I", CSRC, "-o", exe, src], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    vals = {"off": {}, "desc": {}}
    for line in out.splitlines():
        f = line.split()
        if f[0] == "off":
            vals["off"][(int(f[1]), int(f[2]))] = int(f[3])
        elif f[0] == "desc":
            vals["desc"][int(f[1])] = int(f[2])
        elif f[0] == "idesc":
            vals["idesc"] = int(f[1])
        elif f[0] == "smem":
            vals["smem"] = tuple(int(x) for x in f[1:])
    return vals


def bits(v, lo, hi):
    return (v >> lo) & ((1 << (hi - lo + 1)) - 1)


def test_swizzled_tile_is_a_permutation_of_16_byte_slots(values):
    off = values["off"]
    assert len(off) == 128 * 8
    slots = sorted(off.values())
    assert slots == [16 * i for i in range(1024)]   # every slot of the 16 KB tile once


def test_swizzle_matches_the_hardware_xor(values):
    # 128-byte swizzle: the 16-byte chunk index (address bits 4-6) is the
    # logical chunk XOR address bits 7-9 (the row within its 8-row group)
    for (r, c), o in values["off"].items():
        assert o // 128 == r
        assert bits(o, 4, 6) == c ^ bits(o, 7, 9)


def test_staging_stores_are_conflict_free(values):
    # the kernel's mapping: thread t, step i -> q = t + 128 i, row q >> 3,
    # chunk q & 7; each 8-thread phase of a 16-byte store must hit 8
    # different 16-byte bank groups
    off = values["off"]
    for i in range(8):
        for t0 in range(0, 128, 8):
            groups = set()
            for t in range(t0, t0 + 8):
                q = t + 128 * i
                groups.add((off[(q >> 3, q & 7)] // 16) % 8)
            assert len(groups) == 8


def test_matrix_descriptor_fields(values):
    for a, d in values["desc"].items():
        assert bits(d, 0, 13) == (a >> 4) & 0x3FFF
        assert bits(d, 14, 15) == 0
        assert bits(d, 16, 29) == 1            # leading byte offset (unused when swizzled)
        assert bits(d, 32, 45) == 1024 >> 4    # 8-row groups 1024 bytes apart
        assert bits(d, 46, 47) == 1            # descriptor version
        assert bits(d, 49, 51) == 0 and bits(d, 52, 52) == 0
        assert bits(d, 61, 63) == 2            # 128-byte swizzle


def test_instruction_descriptor_fields(values):
    d = values["idesc"]
    assert bits(d, 0, 3) == 0                  # dense, no saturation
    assert bits(d, 4, 5) == 1                  # FP32 accumulator
    assert bits(d, 7, 9) == 1 and bits(d, 10, 12) == 1   # A, B BF16
    assert bits(d, 13, 16) == 0                # no negation, both K-major
    assert bits(d, 17, 22) == 128 >> 3 and bits(d, 24, 28) == 128 >> 4
    assert bits(d, 23, 23) == 0 and bits(d, 29, 31) == 0


def test_shared_memory_budget(values):
    smem, stages, tile_a, tile_b, cols = values["smem"]
    assert tile_a == tile_b == 128 * 64 * 2
    # stages, barriers and the TMEM address slot behind up to 1023 bytes of
    # alignment slack, within one block's 227 KB; 128 TMEM columns (power of
    # two, at least 32) hold the 128 x 128 FP32 accumulator
    assert stages * (tile_a + tile_b) + 1023 + 8 * stages + 4 <= smem <= 232448
    assert cols == 128 and cols & (cols - 1) == 0
