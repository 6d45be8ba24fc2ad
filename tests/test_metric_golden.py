"""The benchmark's metric against the worked example the paper prints
(Sec. 4.2.2: B_node = 2 q s_d, P_B = B_node P_LUPS, U_B = P_B / B_peak, with
C = 0.131 / 0.263 for the Titan Xp's 547.68 GB/s and two rows of Table 2)."""
import os

import numpy as np

import bench

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "metric_titanxp.txt")
TITAN_XP_GBS = 547.68


def test_bytes_per_node_and_utilisation_match_paper():
    rows = np.loadtxt(GOLDEN)
    for s_d, b_node, c, glups, gbs, u_b in rows:
        prec = {4: "f32", 8: "f64"}[int(s_d)]
        assert bench.node_bytes(prec) == int(b_node)
        # U_B = C * P_GLUPS with C = B_node / B_peak (printed to 3 digits)
        assert round(bench.node_bytes(prec) / TITAN_XP_GBS, 3) == c
        # P_B = B_node * P_LUPS: the printed GB/s is within rounding of the
        # printed GLUPS (both rounded in the table)
        assert abs(bench.node_bytes(prec) * glups - gbs) <= 0.5 * bench.node_bytes(prec) * 0.01 + 0.5
        assert round(gbs / TITAN_XP_GBS, 3) == u_b


def test_fp16_shifted_bytes_per_node():
    assert bench.node_bytes("f16s") == 36
