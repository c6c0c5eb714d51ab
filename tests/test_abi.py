"""C-ABI library: loads without a GPU, exports every symbol include/*.h
declares, validates arguments on the host before touching the device."""
import ctypes
import dataclasses
import glob
import os
import re

import numpy as np
import pytest

from paper_2511_15629_b300 import build as B
from paper_2511_15629_b300 import esdp as E
from paper_2511_15629_b300 import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return E.load_library()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(esdp_[a-z_0-9]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"esdp_create", "esdp_solve", "esdp_policy", "esdp_bid_curves", "esdp_grad"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(E.EXPORTS) <= names


def test_version(lib):
    assert lib.esdp_version() == 1


def test_struct_layout_matches_header():
    # 10 int32 followed by 5 doubles
    assert ctypes.sizeof(E.Asset) == 10 * 4 + 5 * 8
    assert E.Asset.s_max.offset == 40


def _create(lib, asset, flags=0):
    ctx = ctypes.c_void_p()
    arr = (E.Asset * 1)(asset)
    rc = lib.esdp_create(arr, 1, flags, ctypes.byref(ctx))
    msg = lib.esdp_last_error(ctx).decode() if ctx else ""
    if ctx:
        lib.esdp_destroy(ctx)
    return rc, msg


@pytest.mark.parametrize("field,value,needle", [
    ("A", 7, "A must equal"), ("n_modes", 3, "n_modes"), ("eta_c", 1.5, "efficiencies"),
    ("eta_d", 0.0, "efficiencies"), ("policy_bytes", 3, "policy_bytes"), ("N", 1, "N >= 2"),
    ("s0", 10_000, "s0"), ("K", 200, "supported"), ("s_max", -1.0, "s_max"),
    ("N", (1 << 24) + 1, "2^24"),
])
def test_invalid_asset_rejected_on_host(lib, field, value, needle):
    a = E.asset_from_instance(I.random_instance(0, 3, 20, 4, 2, 3))
    setattr(a, field, value)
    rc, msg = _create(lib, a)
    assert rc == E.ESDP_EINVAL
    assert needle in msg


def test_null_arguments(lib):
    assert lib.esdp_create(None, 1, 0, None) == E.ESDP_EINVAL
    assert lib.esdp_solve(None, None, None, None, None, None, None) == E.ESDP_EINVAL
    assert lib.esdp_grad(None, 0, None, None, None, None, None, None, None, None, None,
                         None) == E.ESDP_EINVAL
    assert lib.esdp_objective(None, 0, None, None, None) == E.ESDP_EINVAL
    assert lib.esdp_bids_at(None, 0, 1, 2, 0, None, None, None, None, None, None) == E.ESDP_EINVAL
    assert lib.esdp_bid_curves_packed(None, 0, 1, 2, None, None, None, 0, None) == E.ESDP_EINVAL
    lib.esdp_destroy(None)


def test_allocation_failure_injection(lib, monkeypatch):
    monkeypatch.setenv("ESDP_FAIL_ALLOC", "1")
    a = E.asset_from_instance(I.random_instance(0, 3, 20, 4, 2, 3))
    rc, msg = _create(lib, a)
    assert rc == E.ESDP_ENOMEM and "injected" in msg


# ------------------------------------------------ stagewise-independent path

def test_iid_struct_layout_matches_header():
    # 4 int32 followed by 4 doubles
    assert ctypes.sizeof(E.IidProblemC) == 4 * 4 + 4 * 8
    assert E.IidProblemC.s_max.offset == 16


def _golden(name):
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def test_iid_action_grid_matches_tables_and_oracle(lib):
    """The library's eq. 13 grid (computed on the host, no GPU) has the
    action counts of Tables I and III and the oracle's levels."""
    import math
    from oracle import oracle as O
    from paper_2511_15629_b300 import instances as I
    eta = math.sqrt(0.85)
    for dur, delta, S, P in _golden("table3_grid_sizes.txt"):
        prob = I.IidProblem("t3", 1, int(S), 1, dur, 1.0, eta, None, None)
        p = E.iid_actions(prob)
        assert len(p) == int(P)
        ref, _, _ = O.paper_action_grid(1.0, dur / (S - 1), eta)
        np.testing.assert_allclose(p, ref, rtol=0, atol=1e-12)
    for delta, P in _golden("table1_action_counts.txt"):
        prob = I.IidProblem("t1", 1, int(round(4.0 / delta)) + 1, 1, 4.0, 1.0, eta, None, None)
        assert len(E.iid_actions(prob)) == int(P)


def test_iid_rejects_bad_problems(lib):
    from paper_2511_15629_b300 import instances as I
    prob = I.iid_problem(1, 3, 11, 4, 1.0)
    for field, value in [("eta", 1.5), ("S", 1), ("R", 0), ("R", 4097), ("policy_bytes", 3),
                         ("tau", 0.0)]:
        bad = dataclasses.replace(prob, **{field: value})
        with pytest.raises(E.EsdpError) as ei:
            E.solve_iid(bad, policy_bytes=getattr(bad, "policy_bytes"))
        assert ei.value.code == E.ESDP_EINVAL
