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


def _write_profile(path, digest, packets, nbytes):
    with open(path, "w") as f:
        f.write("# DRAM traffic\n\nkernel_sources_sha256: `%s`\npackets: `%d`\ndram_bytes_per_launch: `%d`\n"
                % (digest, packets, nbytes))


def test_traffic_is_reported_only_for_the_profiled_code_and_size(tmp_path, monkeypatch):
    n = 16_777_216
    # a profile taken on the current code at n packets is reported at n packets only
    prof = os.path.join(tmp_path, "prof.md")
    _write_profile(prof, bench.kernel_digest(), n, 393_098_752)
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", prof)
    assert bench.traffic_from_profile(n) == 393_098_752
    assert bench.traffic_from_profile(n // 2) is None               # another packet count
    # the committed profile parses, whether or not it matches the current code
    kv = bench.read_profile_fields(os.path.join(ROOT, "profiles", "k_tc256_classify_bf16_dram_512k_16M.md"))
    assert int(kv["packets"]) == n and int(kv["dram_bytes_per_launch"]) >= 20 * n  # >= 20 B/packet of HBM
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
    assert bench.traffic_from_profile(n) is None
