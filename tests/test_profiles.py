"""The committed stencil profile's DRAM-traffic record belongs to the current kernel
sources: bench.py reports roofline.traffic from it only while the SHA-256 of the stencil
sources matches the one recorded with the ncu counters (a changed kernel needs a new
capture), and every profile summary names the command that made it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_matches_kernel_sources():
    sys.path.insert(0, ROOT)
    import bench

    t = bench.recorded_traffic()
    assert t is not None, "stencil sources changed since profiles/hop_f32_24x24x24x48_full.md was captured"
    # DRAM bytes per launch at 32^3x64 within a few per cent of the algorithmic 956.3 MB
    assert 0.9 * 956.3e6 < t < 1.05 * 956.3e6


def test_profiles_name_their_commands():
    d = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(d)):
        if f.endswith(".md"):
            txt = open(os.path.join(d, f)).read()
            assert "bench.py" in txt or "python" in txt, f
