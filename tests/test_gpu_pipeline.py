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


def run_gpu(ref, precision, nsteps, rtol, refine=False):
    p = ref["p"]
    ctx = context(p, precision, ref["o"].dt)
    ctx.set_sources(ref["tables"])
    ctx.em_steps(nsteps)
    E, H = read_eh(ctx)
    Q = ctx.read(api.COSIM_F_Q)
    tot = ctx.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER)
    ctx.thermal_steps(p.thermal_steps)
    T = ctx.read(api.COSIM_F_T)
    rep = ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=rtol, refine=refine,
                           inner_rtol=1e-4 if refine else 0.0)
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


def test_config1_precision_ladder(ref10k):
    """Precision ladder on the 32x32x16 package after 10^4 EM steps: FP64
    kernels, FP32 kernels (FP64 Joule totals and CG dots), and FP32 kernels
    with the stress solve in FP64 iterative refinement. Prints the per-field
    relative L2 error of each against the FP64 oracle and of FP32 against the
    FP64 GPU run; the refined FP32 solve must reach the FP64 bars for the
    displacement and von Mises stress (1e-6 at a 1e-9 true residual)."""
    runs = {"fp64": run_gpu(ref10k, FP64, 10_000, 1e-9),
            "fp32": run_gpu(ref10k, FP32, 10_000, 1e-6),
            "fp32+ir": run_gpu(ref10k, FP32, 10_000, 1e-9, refine=True)}
    ref_u = interleaved_to_soa(ref10k["res"]["u"])

    def errors(g, r):
        return {"E": field_rel_l2(g["E"], r["E"])[0], "H": field_rel_l2(g["H"], r["H"])[0],
                "Q": rel_l2(g["Q"], r["Q"]), "P_total": abs(g["total"] / r["total"] - 1),
                "dT": rel_l2(g["T"] - 300, r["T"] - 300), "u": rel_l2(g["u"], r["u"]),
                "vm": rel_l2(g["vm"], r["vm"])}

    oracle_ref = dict(E=ref10k["E"], H=ref10k["H"], Q=ref10k["Q"], total=ref10k["total"], T=ref10k["T"],
                      u=ref_u, vm=ref10k["res"]["vm"])
    table = {k: errors(g, oracle_ref) for k, g in runs.items()}
    table["fp32 vs fp64 GPU"] = errors(runs["fp32"], runs["fp64"])
    cols = list(table["fp64"].keys())
    print("\nprecision ladder, relative L2 vs the FP64 oracle (10^4 EM steps):")
    print("| run | " + " | ".join(cols) + " | CG iters | refine steps |")
    for k, e in table.items():
        rep = runs[k]["rep"] if k in runs else None
        extra = f" {rep['iters']} | {rep.get('refine_steps', 0)} |" if rep else " | |"
        print(f"| {k} | " + " | ".join(f"{e[c]:.1e}" for c in cols) + " |" + extra)
    assert max(table["fp64"].values()) < 1e-6
    assert max(table["fp32"][c] for c in ("E", "H", "Q", "P_total", "dT")) < 1e-4
    assert table["fp32+ir"]["u"] < 1e-6 and table["fp32+ir"]["vm"] < 1e-6
    assert runs["fp32+ir"]["rep"]["relres"] <= 1e-9
