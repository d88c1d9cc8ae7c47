"""FGMRES iteration counts on the GPU against the oracle's stored counts, at 132k DoFs.

Two 2D 128^2 configurations, whose oracle counts are stored by committed scripts that call
only oracle/ (tests/golden/make_*.py):

  * the 2D multi-sinker configuration (5 levels, 8 sinkers, DR 1e6, gamma 1, 1e2, 1e4,
    P1, V-cycle, rtol 1e-8): the FP64 GPU solve needs exactly the oracle's iteration
    count (within one at gamma 1e4); the mixed solve at most 2 more where the FP32 cycle is within its range
    (eps32 gamma / mu_min below 0.1, i.e. gamma 1 and 1e2 here);
  * the AL column of Table vanka (Sec. 5.2.3: 4 levels, P2 with gamma 100, F-cycle, 1e6
    residual reduction, 1/6/24 sinkers, DR 1e4..1e8): the FP64 GPU solve needs the
    oracle's count (within 2 at DR 1e8, where the patch inverses' cond * eps difference
    can move the step at which the tolerance is crossed).  How the stored counts compare
    with the printed column is pinned on the CPU (tests/test_oracle_pins.py).

The file name sorts after the other GPU tests so that they run first."""
import os

import pytest

from gpu_helpers import context  # noqa: F401
from synthetic import problems as P

from paper_2107_00820_gb300 import alstokes as A  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        out.append(line.split())
    return out


@pytest.mark.parametrize("row", _rows("sinker2d_128_oracle.txt"), ids=lambda r: "gamma" + r[0])
def test_sinker2d_128_counts_equal_the_oracle(row):
    gamma, its_oracle = float(row[0]), int(row[1])
    pb = P.sinker_problem(2, 128, 5, 8, 0.1, 200.0, 1e6, 10.0, gamma, 0)
    ctx = context(pb, sweeps=5, rtol=1e-8, maxit=300)
    _, _, info = ctx.solve(pb.f, pb.u_bc)
    ctx.close()
    # gamma 1e4: the patch inverses' cond * eps (about 2e4 gamma / mu_min * 1e-16 = 2e-5)
    # separates the two sides enough to move the crossing of the tolerance by one step
    slack = 0 if gamma <= 1e2 else 1
    assert info.converged and abs(info.iterations - its_oracle) <= slack, (info.iterations, its_oracle)
    if 2.0 ** -24 * gamma / 1e-3 < 0.1:
        mixed = context(pb, sweeps=5, rtol=1e-8, maxit=300, mode=A.ALS_MODE_MIXED)
        _, _, im = mixed.solve(pb.f, pb.u_bc)
        mixed.close()
        assert im.converged and im.iterations <= its_oracle + 2, (im.iterations, its_oracle)


@pytest.mark.parametrize("row", [r for r in _rows("table_vanka_oracle.txt") if float(r[1]) <= 1e8],
                         ids=lambda r: f"sinkers{r[0]}-DR{r[1]}")
def test_table_vanka_al_column_counts_equal_the_oracle(row):
    s, dr, its_oracle = int(row[0]), float(row[1]), int(row[2])
    pb = P.sinker_problem(2, 128, 4, s, 0.1, 200.0, dr, 10.0, 100.0, 0)
    ctx = context(pb, sweeps=5, rtol=1e-6, maxit=300, schur=A.ALS_SCHUR_P2, cycle=A.ALS_CYCLE_F)
    _, _, info = ctx.solve(pb.f, pb.u_bc)
    ctx.close()
    slack = 0 if dr <= 1e6 else 2
    assert info.converged and abs(info.iterations - its_oracle) <= slack, (info.iterations, its_oracle)
