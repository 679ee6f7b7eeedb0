"""The benchmark's measurement plumbing on CPU: the algorithmic FLOP count of the paper's network
(§6.1: 7 -> 512, six residual blocks of two 512 x 512 layers, 512 -> T) and the rule that the
profiled DRAM traffic is reported only for the kernel code and packet count it was captured on."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_flops_per_packet_of_the_paper_network():
    # layer 0: 7 x 512 multiply-adds; 12 hidden layers of 512 x 512; output 512 x T
    assert bench.flops_per_packet(25) == 2 * (7 * 512 + 12 * 512 * 512 + 512 * 25) == 6_324_224
    assert bench.flops_per_packet(1) - bench.flops_per_packet(0) == 2 * 512


def test_traffic_is_reported_only_for_the_profiled_code_and_size(tmp_path, monkeypatch):
    n = 16_777_216
    v = bench.traffic_from_profile(n)
    assert v is not None and 335_544_320 <= v < 2 * 335_544_320  # at least the 20 B/packet of HBM
    assert bench.traffic_from_profile(n // 2) is None               # another packet count
    # a comment edit keeps the digest; a code edit changes it
    src = os.path.join(tmp_path, "k.cu")
    with open(src, "w") as f:
        f.write('// a comment\nint f(int x) { return x + 1; }  /* another */\nconst char *s = "a // b";\n')
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [src])
    d0 = bench.kernel_digest()
    with open(src, "w") as f:
        f.write('// changed comment\nint f(int x)  {  return x + 1; }\n/* gone */ const char *s = "a // b";\n')
    assert bench.kernel_digest() == d0
    with open(src, "w") as f:
        f.write('// a comment\nint f(int x) { return x + 2; }  /* another */\nconst char *s = "a // b";\n')
    assert bench.kernel_digest() != d0
    with open(src, "w") as f:
        f.write('// a comment\nint f(int x) { return x + 1; }  /* another */\nconst char *s = "a // c";\n')
    assert bench.kernel_digest() != d0
    # and the traffic figure disappears when the profiled digest no longer matches
    prof = os.path.join(tmp_path, "prof.md")
    shutil.copy(bench.TRAFFIC_PROFILE, prof)
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", prof)
    assert bench.traffic_from_profile(n) is None
