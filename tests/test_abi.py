"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/lbm.h declares, its velocity tables match Table A.1, its
parameter mapping agrees with the oracle's, and calls that need a device fail
with a status instead of crashing when none is present."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_14505_gb300 import build as cuda_build
from paper_2605_14505_gb300 import lbm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table_a1_stencils.txt")


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return lbm.load_library()


def test_library_exports_every_declared_symbol(lib):
    names = lbm.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps each of them
    assert set(names) <= set(lbm._SIGS), set(names) - set(lbm._SIGS)


def test_velocity_sets_match_table_a1(lib):
    from fractions import Fraction

    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, cs2, m, count, w = line.split()
            rows.append((int(name[3:]), float(Fraction(cs2)), int(m), int(count), float(Fraction(w))))
    for q in (7, 15, 19, 27):
        e, w, cs2 = lbm.lbm_velocity_set(q)
        assert len(w) == q
        m2 = (e ** 2).sum(axis=1)
        for qq, c2, m, count, wt in rows:
            if qq != q:
                continue
            assert abs(cs2 - c2) < 1e-16
            assert (m2 == m).sum() == count
            assert np.all(np.abs(w[m2 == m] - wt) < 1e-16)
        # slot 0 is rest; slots 2m-1 and 2m are opposite
        assert np.all(e[0] == 0)
        for i in range(1, q, 2):
            assert np.all(e[i] == -e[i + 1])
        assert len({tuple(v) for v in e}) == q


def test_invalid_velocity_set(lib):
    with pytest.raises(lbm.LbmError):
        lbm.lbm_velocity_set(9)


@pytest.mark.parametrize("n,pair,Re,Fr,Pr", [(32, "27x19", 100, 0.5, 1.0), (128, "19x7", 400, 0.1, 1.0),
                                             (256, "27x19", 800, 0.1, 1.0), (64, "19x7", 200, 1.0, 0.7)])
def test_physics_mapping_agrees_with_oracle(lib, n, pair, Re, Fr, Pr):
    p = lbm.lbm_params_from_physics(n, n, n, pair, "sc", Re, Fr, Pr, 0.04)
    qf, qg = lbm.PAIR_Q[lbm.PAIRS[pair]]
    o = O.params_from_physics(n, qf, qg, "sc", Re, Fr, Pr, 0.04)
    for key in ("tau_f", "tau_g", "G", "beta", "rho0", "sc_shift"):
        assert abs(getattr(p, key) - getattr(o, key)) <= 1e-14 * max(1.0, abs(getattr(o, key))), key
    assert p.scalar_mode == o.scalar_mode == 0


def test_mapping_rejects_bad_numbers(lib):
    for args in [(0, 0, 0, 0, 0, 100, 0.5, 1, 0.04), (32, 32, 32, 9, 0, 100, 0.5, 1, 0.04),
                 (32, 32, 32, 0, 0, -1, 0.5, 1, 0.04), (32, 32, 32, 0, 0, 100, 0.0, 1, 0.04),
                 (32, 32, 32, 0, 0, 100, 0.5, 1, 0.0)]:
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_params_from_physics(*args)
        assert ei.value.code == -1


def test_unstratified_mapping(lib):
    p = lbm.lbm_params_from_physics(32, 32, 32, 0, 0, 100, float("inf"), 1, 0.04)
    assert p.G == 0.0 and p.beta == 0.0


def test_null_handle_is_an_error_not_a_crash(lib):
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_destroy(None) == 0
    assert "null" in lbm.lbm_last_error()


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="only meaningful without a GPU")
def test_create_without_device_reports_cuda_error(lib):
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(8, 8, 8, 0, 0, 100, 0.5, 1, 0.04)
    assert ei.value.code == -3
