"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/mw3.h declares, and its host-side set-up (grids, bases, spectral bounds,
diatomic reference energy) agrees with the oracle. No device work: contexts are
created with device = -1 (set-up mathematics only)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import propagate as P
from oracle.hamiltonian import GridHamiltonian

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "mw3.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(mw3_[a-z_0-9]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    from paper_2412_10167_gb300 import mw3
    syms = declared_symbols()
    assert len(syms) >= 25
    raw = ctypes.CDLL(mw3._LIB_PATH)
    for s in syms:
        assert hasattr(raw, s), s
    # the binding wraps every declared entry point under the same name
    assert set(syms) <= set(mw3.EXPORTED) | {"mw3_pot_fn", "mw3_alloc_fn", "mw3_free_fn"}


@pytest.mark.parametrize("name", list(W.SMALL))
def test_host_setup_matches_oracle(name):
    from paper_2412_10167_gb300 import mw3
    cfg = W.SMALL[name]
    pr = mw3.Propagator(cfg, device=-1)
    E0, dE = pr.spectral_range()
    H = GridHamiltonian(cfg)
    _, info = P.initial_packet(H, cfg["packet"])
    np.testing.assert_allclose(E0, H.E0, rtol=1e-14)
    np.testing.assert_allclose(dE, H.dE, rtol=1e-14)
    assert abs(pr.reference_energy() - info["E_v0j0"]) < 1e-13
    assert pr.shape == H.shape


@pytest.mark.parametrize("name", ["c2s", "c3s", "c4s"])
def test_product_stencil_columns_host(name):
    """Plane-major product-channel sums (tuning key prod_gather, the default): the set-up
    gathers each distinct grid column of the 4 x 4 interpolation stencils once; their
    number equals the count from the oracle's own product quadrature stencils (Section
    2.4; points beyond the grid are column 0 with weight 0 on both sides)."""
    from paper_2412_10167_gb300 import mw3
    from oracle import products as PR
    cfg = W.SMALL[name]
    pr = mw3.Propagator(cfg, device=-1)
    H = GridHamiltonian(cfg)
    pa = PR.ProductAnalysis(H, cfg["analysis"]["products"])
    cols = {int(k) * H.NR + int(m) for n in range(len(pa.R)) for k in pa.kidx[n] for m in pa.midx[n]}
    assert pr.get_tuning("prod_gather") == 1
    assert pr.get_tuning("prod_points") == len(cols)
    assert pr.set_tuning("prod_gather", 0) is None and pr.get_tuning("prod_gather") == 0


def test_error_paths_host_only():
    from paper_2412_10167_gb300 import mw3
    lib = mw3.lib
    h = ctypes.c_void_p()
    assert lib.mw3_create(ctypes.byref(h), -1, 7) == -1          # bad precision
    assert lib.mw3_create(ctypes.byref(h), -1, mw3.MW3_FP64) == 0
    # out of order: analysis before grid
    d = mw3.mw3_analysis_desc(6.0, 0.01, 0.05, 10, 10.5, -1, 0, 0)
    assert lib.mw3_set_analysis(h, ctypes.byref(d)) == -7
    assert lib.mw3_propagate(h, 10) == -7
    # bad grid: odd NR, radix 7
    J = (ctypes.c_int * 1)(0)
    for NR in (63, 14):
        g = mw3.mw3_grid_desc(NR, 0.5, 14.0, 48, 0.5, 10.0, 24, (ctypes.c_double * 3)(1, 2, 1),
                              1, J, 0, 1)
        assert lib.mw3_grid(h, ctypes.byref(g)) == -1
        assert b"NR" in lib.mw3_last_error(h)
    assert lib.mw3_set_tuning(h, b"kb", 0) == -1
    assert lib.mw3_set_tuning(h, b"nonsense", 1) == -1
    assert lib.mw3_set_tuning(h, b"use_tc", 1) == -1              # needs MW3_MIXED
    assert lib.mw3_set_tuning(h, b"kb", 48) == 0 and lib.mw3_get_tuning(h, b"kb") == 48
    # bounded-wait poll limit of the tile-major angular step: 0..2^22, default 2^22
    assert lib.mw3_get_tuning(h, b"tc_wait_limit") == 1 << 22
    assert lib.mw3_set_tuning(h, b"tc_wait_limit", -1) == -1
    assert lib.mw3_set_tuning(h, b"tc_wait_limit", (1 << 22) + 1) == -1
    assert lib.mw3_set_tuning(h, b"tc_wait_limit", 0) == 0 and lib.mw3_get_tuning(h, b"tc_wait_limit") == 0
    lib.mw3_destroy(h)
    assert lib.mw3_status_string(-4) == b"propagation diverged"


def test_nan_potential_rejected():
    from paper_2412_10167_gb300 import mw3
    cfg = W.SMALL["c1"]
    ctx = mw3.mw3_create(-1, mw3.MW3_FP64)
    g = cfg["grid"]
    mw3.mw3_grid(ctx, g["NR"], g["Rmin"], g["Rmax"], g["nr"], g["rmin"], g["rmax"], g["ngamma"],
                 (1837.0, 3671.0, 1837.0), [0], 0, 1)
    V = np.zeros((1, 1, g["ngamma"], g["nr"], g["NR"]))
    V[0, 0, 3, 4, 5] = np.nan
    with pytest.raises(mw3.MW3Error) as e:
        mw3.mw3_load_potential_grid(ctx, V, 0.1, 0.1, 0.2)
    assert e.value.code == -9
    mw3.mw3_destroy(ctx)


def test_leps_callback_matches_oracle_surface():
    from paper_2412_10167_gb300 import mw3
    from oracle import pes
    from oracle.units import AMU, EV
    cfg = W.C3
    masses = [m * AMU for m in cfg["masses_u"]]
    p = mw3.mw3_leps_params()
    p.D = W.LEPS_H3["D_eV"] * EV
    p.beta, p.re, p.delta = W.LEPS_H3["beta"], W.LEPS_H3["re"], W.LEPS_H3["delta"]
    p.masses = (ctypes.c_double * 3)(*masses)
    ts = W.TWO_STATE
    p.two_state = 1
    p.bump, p.bump_r0, p.bump_w2 = ts["bump_eV"] * EV, ts["bump_r0"], ts["bump_w2"]
    p.coup, p.coup_R0, p.coup_r0, p.coup_w2 = ts["coup_eV"] * EV, ts["coup_R0"], ts["coup_r0"], ts["coup_w2"]
    out = (ctypes.c_double * 4)()
    rng = np.random.default_rng(5)
    for _ in range(40):
        r, R, cg = rng.uniform(0.5, 8), rng.uniform(0.5, 12), rng.uniform(-1, 1)
        assert mw3.lib.mw3_pes_leps(r, R, cg, out, ctypes.cast(ctypes.pointer(p), ctypes.c_void_p)) == 0
        ref = pes.potential_matrix(r, R, cg, masses, cfg["pes"])
        np.testing.assert_allclose(np.array(out[:]).reshape(2, 2), ref, rtol=1e-13, atol=1e-15)
