"""The whole hot path on the 32x32x16 package, CUDA path vs the FP64 oracle:
EM burst with Joule accumulation -> burst-averaged source -> thermal steps ->
clamped-bottom thermoelastic solve.

Bars: FP64 kernels, 1000 EM steps: E, H, Q within 1e-10 (rounding order);
FP32 kernels, 10^4 EM steps: E, H and the temperature rise T - T_init within
1e-4 relative L2; displacement and von Mises within 1e-6 once CG reaches a
1e-9 relative residual (FP64 path)."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2603_07038_b300 import cosim as api
from tests.gpu_helpers import FP32, FP64, context, field_rel_l2, interleaved_to_soa, read_eh, rel_l2
from workloads import constraints as BC

pytestmark = pytest.mark.gpu


def run_oracle(nsteps):
    p = W.tiny_package()
    o = oracle.OracleSim(p)
    tables = p.source_tables(o.dt, nsteps)
    o.set_sources(tables)
    o.em_steps(nsteps)
    E, H, Q = [e.copy() for e in o.E], [h.copy() for h in o.H], o.Q.copy()
    tot = o.joule_finalize_avg_power()
    o.thermal_steps(p.thermal_steps)
    res = o.stress_solve(BC.clamped_bottom(p), 300.0, rtol=1e-13)
    return dict(p=p, o=o, tables=tables, E=E, H=H, Q=Q, total=tot, T=o.T.copy(), res=res)


def run_gpu(ref, precision, nsteps, rtol):
    p = ref["p"]
    ctx = context(p, precision, ref["o"].dt)
    ctx.set_sources(ref["tables"])
    ctx.em_steps(nsteps)
    E, H = read_eh(ctx)
    Q = ctx.read(api.COSIM_F_Q)
    tot = ctx.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER)
    ctx.thermal_steps(p.thermal_steps)
    T = ctx.read(api.COSIM_F_T)
    rep = ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=rtol)
    u = np.stack([ctx.read(api.COSIM_F_UX + c) for c in range(3)])
    vm = ctx.read(api.COSIM_F_VM)
    ctx.close()
    return dict(E=E, H=H, Q=Q, total=tot, T=T, u=u, vm=vm, rep=rep)


@pytest.fixture(scope="module")
def ref1000():
    return run_oracle(1000)


@pytest.fixture(scope="module")
def ref10k():
    return run_oracle(10_000)


def test_config1_fp64_full_path(ref1000):
    g = run_gpu(ref1000, FP64, 1000, 1e-9)
    for a in range(3):
        assert rel_l2(g["E"][a], ref1000["E"][a]) < 1e-10
        assert rel_l2(g["H"][a], ref1000["H"][a]) < 1e-10
    assert rel_l2(g["Q"], ref1000["Q"]) < 1e-10
    assert abs(g["total"] / ref1000["total"] - 1) < 1e-10
    assert rel_l2(g["T"] - 300, ref1000["T"] - 300) < 1e-9
    assert g["rep"]["relres"] <= 1e-9
    assert rel_l2(g["u"], interleaved_to_soa(ref1000["res"]["u"])) < 1e-6
    assert rel_l2(g["vm"], ref1000["res"]["vm"]) < 1e-6


def test_config1_fp32_10k_steps(ref10k):
    """E and H are compared as vector fields (all components together); the
    per-component error norms are measured against the same field norm. The
    port's field is vertical (|Ez| is ~400x |Ex| here), so a component-wise
    ratio would divide cross-component rounding by a tiny norm."""
    g = run_gpu(ref10k, FP32, 10_000, 1e-6)
    eE, perE = field_rel_l2(g["E"], ref10k["E"])
    eH, perH = field_rel_l2(g["H"], ref10k["H"])
    errs = {"E": eE, "H": eH, "Q": rel_l2(g["Q"], ref10k["Q"]), "dT": rel_l2(g["T"] - 300, ref10k["T"] - 300)}
    print("FP32 10^4-step relative L2 errors:", {k: f"{v:.2e}" for k, v in errs.items()},
          "E components", [f"{v:.1e}" for v in perE], "H components", [f"{v:.1e}" for v in perH],
          "component-wise Ex", f"{rel_l2(g['E'][0], ref10k['E'][0]):.1e}")
    assert max(errs.values()) < 1e-4, errs
    assert np.max(ref10k["T"] - 300) > 0  # the burst did heat the package


def test_config1_fp64_10k_steps(ref10k):
    g = run_gpu(ref10k, FP64, 10_000, 1e-9)
    for a in range(3):
        assert rel_l2(g["E"][a], ref10k["E"][a]) < 1e-9
        assert rel_l2(g["H"][a], ref10k["H"][a]) < 1e-9
    assert rel_l2(g["T"] - 300, ref10k["T"] - 300) < 1e-9
    assert rel_l2(g["u"], interleaved_to_soa(ref10k["res"]["u"])) < 1e-6
    assert rel_l2(g["vm"], ref10k["res"]["vm"]) < 1e-6
