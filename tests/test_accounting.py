"""The FLOP/byte accounting against numbers the paper prints (CPU only)."""
import pytest

from paper_2202_12477_gb300 import accounting as acc


def test_fom_over_throughput_matches_nekbone_count():
    """N=7, 50^3 elements, one V100: FOM 657.6 GFLOPS (Fig. SummitScaling, FOM
    panel) and 3.36e9 DOF*it/s (throughput panel). Their ratio is the NekBone
    FLOP count per DOF per iteration with E = all elements (Eq. nekbone_flops)."""
    E, N = 50 ** 3, 7
    NG = acc.box_dofs(N, 50, 50, 50)
    assert NG == 42508549
    per_dof = acc.nekbone_flops(E, N) / NG
    assert abs(per_dof - 657.6e9 / 3.36e9) / per_dof < 2e-3


def test_fom_over_throughput_n15():
    """N=15, 24^3: FOM 1051.5 GFLOPS and 3.80e9 DOF*it/s on one V100."""
    E, N = 24 ** 3, 15
    NG = acc.box_dofs(N, 24, 24, 24)
    assert NG == 46268279
    per_dof = acc.nekbone_flops(E, N) / NG
    assert abs(per_dof - 1051.5e9 / 3.80e9) / per_dof < 5e-3


@pytest.mark.parametrize("N,gflops,B,frac", [(7, 1128.6, 820e9, 0.886), (15, 2101.4, 820e9, 0.907)])
def test_paper_operator_roofline_fraction(N, gflops, B, frac):
    """Eq. op_perf with the plotted V100 stream rate (820 GB/s) against the V100
    operator figures (Fig. AxOperator): ~0.89 (N=7) and ~0.91 (N=15)."""
    R = acc.paper_roofline(N, B) / 1e9
    assert abs(gflops / R - frac) < 0.005


def test_flop_counts_per_element():
    assert acc.op_flops(1, 7) == 12 * 8 ** 4 + 18 * 8 ** 3 == 58368
    assert acc.op_local_flops(1, 1) == 12 * 16 + 15 * 8
    assert acc.hipbone_cg_flops(1, 7) == 12 * 8 ** 4 + 19 * 8 ** 3 + 10 * 7 ** 3


def test_byte_models():
    assert acc.ax_min_bytes(10, 20, 8) == 16 * 10 + 52 * 20
    assert acc.ax_min_bytes(10, 20, 4) == 8 * 10 + 28 * 20
    assert acc.paper_op_bytes(10, 20) == 8 * 10 + 68 * 20
    assert acc.paper_cg_bytes(10, 20) == 108 * 10 + 80 * 20
