"""The committed ncu summaries under profiles/ that bench.py reads `roofline.traffic` from:
each names the kernel sources it was taken on and a DRAM traffic per step within 10 % of
the workload's algorithmic bytes, and its commands run committed files only."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")

# summary -> algorithmic bytes of one step of its bench workload
ALGORITHMIC = {
    "step_std_f32_4096.md": 77 * 4096 * 4096,         # 9x4 read + 9x4 write + KL + flag
    "step_aar_std_f32_4096.md": 79 * 4096 * 4096,     # + region byte read and written
    "batch_multi_f32_64lattices.md": 77 * 15769600,   # the 64-lattice batch's cells
    "step_std_f16dev_8192.md": 41 * 8192 * 8192,      # 9x2 read + 9x2 write + KL + flag
}


@pytest.mark.parametrize("name", sorted(ALGORITHMIC))
def test_traffic_summary_is_well_formed(name):
    with open(os.path.join(PROFILES, name)) as fh:
        txt = fh.read()
    assert re.search(r"kernel_sources_sha256_16:\s*[0-9a-f]{16}\b", txt)
    m = re.search(r"dram_bytes_per_step:\s*([0-9.eE+]+)", txt)
    assert m, name
    ratio = float(m.group(1)) / ALGORITHMIC[name]
    assert 0.9 <= ratio <= 1.1, (name, ratio)
    assert "--clock-control none" in txt
    for script in re.findall(r"python ([\w./-]+\.py)", txt):
        assert os.path.exists(os.path.join(ROOT, script)), (name, script)


def test_bench_reads_every_traffic_summary():
    with open(os.path.join(ROOT, "bench.py")) as fh:
        src = fh.read()
    for name in ALGORITHMIC:
        assert f'"{name}"' in src, name
