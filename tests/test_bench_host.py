"""Host logic of bench.py: the algorithmic work counts behind its roofline fractions and the
DRAM traffic figures it takes from the committed profiles."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import symmetry  # noqa: E402
from paper_2509_07974_gb300 import ext4pcf  # noqa: E402


def test_reduced_contraction_count_is_the_exchange_map_of_the_symmetry_table():
    """The tensor-core contraction produces, per component mu', the multipoles that the
    identity and the exchange of Theta2 and Theta3 (column 2 of Table tab:4PCFSymm) read:
    counted here from the oracle's map, over the bin pairs Theta2 <= Theta3 and every Theta1."""
    for N in (0, 1, 3, 20):
        reached = 0
        for mup in range(9):
            need = set()
            for mu in range(9):
                for n2 in range(-N, N + 1):
                    for n3 in range(-N, N + 1):
                        if mu == mup:
                            need.add((n2, n3))
                        if symmetry.MU_MAP[mu][2] == mup:
                            need.add(symmetry.n_map(mu, 2, n2, n3))
            reached += len(need)
        for nb in (1, 4, 10):
            pairs = nb * (nb + 1) // 2
            assert bench.reduced_contraction_flop(1, N, nb) == 8 * reached * pairs * nb
    # at the bench's sizes (N = 20, 10 bins) the reduction does 1.74x less work than all ordered triples
    assert abs(bench.contraction_flop(1, 20, 10) / bench.reduced_contraction_flop(1, 20, 10) - 1.7435) < 1e-3


def test_gather_count_follows_the_record_layout():
    """Per pair: one complex multiply-add (8 FLOP) per complex-weighted record entry (G, XX),
    a real weight times a complex power (4 FLOP) per entry of W, XA and WW, one complex
    multiplication (6 FLOP) per power of u up to the largest |n| of the record, and 40 for the
    triple terms."""
    for N in (0, 2, 20, 30):
        lay = ext4pcf.record_layout(1, N)
        top = max(-lay["G"][1], -lay["XX"][1], lay["W"][2] - 1, lay["XA"][2] - 1, lay["WW"][2] - 1)
        want = (8 * (lay["G"][2] + lay["XX"][2]) + 4 * (lay["W"][2] + lay["XA"][2] + lay["WW"][2]) + 6 * top
                + 40)
        assert bench.gather_flop_per_pair(N) == want
    assert bench.gather_flop_per_pair(20) == 2160


def test_traffic_figure_is_used_only_while_the_kernel_source_is_unchanged(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_2509_07974_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "k.cu"
    src.write_text("__global__ void k_kernel() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "k.md").write_text("# a capture\n\n```\ntraffic k_kernel 1.5e9 k.cu %s\n```\n" % sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("k_kernel") == 1.5e9
    assert bench.measured_traffic("other_kernel") is None
    src.write_text("__global__ void k_kernel() { /* changed */ }\n")
    assert bench.measured_traffic("k_kernel") is None


def test_committed_traffic_lines_match_the_current_sources():
    """Every traffic line under profiles/ for the default forms refers to the current source."""
    for kernel in ("gather_kernel", "contract_h16_kernel"):
        assert bench.measured_traffic(kernel) is not None, kernel


def test_clock_summary_reads_median_clock_and_throttle_reasons(tmp_path):
    """The clocks record of the bench line: median SM clock under load, the largest maximum
    clock seen, and every throttle reason that was active in any sample."""
    rows = ["0, 2070, 2070, 610.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1020.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active"]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(path)
    s = cs.summary(2070.0)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 4 and s["power_w_max"] == 1390.0
    # a thermal slowdown in one sample is reported (such a run is re-measured)
    path.write_text(rows[0] + "\n" + rows[0].replace("Not Active, Not Active, Not Active, Not Active",
                                                     "Not Active, Active, Not Active, Not Active") + "\n")
    cs.path = str(path)
    assert bench.ClockSampler.summary(cs, 2070.0)["reasons"] == ["hw_thermal_slowdown"]
    # no samples at all (nvidia-smi missing): the line says so instead of reporting a clock
    cs.path = str(tmp_path / "absent.csv")
    s = cs.summary(2070.0)
    assert s["sm_mhz"] is None and s["reasons"] == ["unsampled"]


def test_pairs_of_mask_counts_the_binned_pairs_of_the_sampled_centres():
    """The pair count behind the oracle's rate: (centre, neighbour) pairs with
    Theta_0 <= separation < Theta_nb, centres the masked galaxies, every galaxy a neighbour,
    against a brute-force count."""
    import numpy as np
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 20, (700, 2))
    pos[5] = pos[4] + (0.5, 0.0)                 # a pair exactly on the inner edge (counted)
    pos[7] = pos[6] + (0.0, 6.0)                 # a pair exactly on the outer edge (not counted)
    edges = np.array([0.5, 1.0, 2.5, 6.0])
    mask = np.zeros(len(pos), np.uint8)
    mask[rng.choice(len(pos), 90, replace=False)] = 1
    mask[[4, 6]] = 1
    d = np.sqrt(((pos[mask.astype(bool)][:, None, :] - pos[None, :, :]) ** 2).sum(-1))
    want = int(((d >= edges[0]) & (d < edges[-1])).sum())
    assert bench.pairs_of_mask(pos, edges, mask) == want
