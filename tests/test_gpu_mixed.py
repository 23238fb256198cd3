"""The mixed-precision path (dense DF contractions as exact BF16 slices on tcgen05 tensor cores, eigensolves and
residual in FP32 with FP64-accurate refinement) against the FP64 GPU path and the oracle: |dE| <= 1e-6 Eh and
max |d grad| <= 1e-6.  Errors are printed.  The split-TF32 mode (precision 1) is rejected by the library."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06149_gb300.synth import Params, make_problem, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osvmbe():
    from paper_2106_06149_gb300 import build, osvmbe as m
    build.build()
    m.load()
    return m


def run(m, p, prm, grad=True):
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    ctx.clusters_build(dp, prm)
    E, El = m.run_energy(ctx, dp, prm)
    out = {"E": E}
    if grad:
        dB = torch.zeros_like(dp.B)
        dF = torch.zeros_like(dp.f_occ)
        ctx.gradient_backward(1.0, dB, dF)
        torch.cuda.synchronize()
        out["dB"] = dB.cpu().numpy().astype(np.float64)
        out["dF"] = dF.cpu().numpy()
    ctx.close()
    return out


@pytest.mark.parametrize("case", ["full", "local", "odd"])
def test_bf16x4_small_matches_fp64_and_oracle(osvmbe, case):
    # "odd": n_vir = 30 (rows not a multiple of four: the FP32 tridiagonalisation's scalar column path) and odd
    # GEMM row lengths (the exact-slice epilogue's element path next to its bulk copies)
    if case == "local":
        p = make_problem(6, 24, 90, geometry="cube", box=7.0, dmin=1.4, radius=4.5, seed=51)
    elif case == "odd":
        p = make_problem(6, 30, 110, seed=53)
    else:
        p = make_problem(6, 40, 150, seed=52)
    base = dict(n_osv_fixed=6, mbe_order=3, r2b=6.0, r3b=5.0, tol=1e-11)
    f = run(osvmbe, p, Params(**base))
    x = run(osvmbe, p, Params(**base, precision=2))
    o = oracle.gradient(p, Params(**base))
    print(f"\nmixed vs fp64: dE = {x['E'] - f['E']:.3e} (E = {f['E']:.6f}); "
          f"max|d dB| = {np.abs(x['dB'] - f['dB']).max():.3e}; max|d dF| = {np.abs(x['dF'] - f['dF']).max():.3e}")
    assert abs(f["E"] - o["E"]) <= 1e-9
    assert abs(x["E"] - f["E"]) <= 1e-6
    assert np.abs(x["dB"] - f["dB"]).max() <= 1e-6
    assert np.abs(x["dF"] - f["dF"]).max() <= 1e-6


def test_split_tf32_mode_is_rejected(osvmbe):
    """Split TF32 with FP32 accumulation misses the 1e-6 Eh bar: the library refuses the mode."""
    p = make_problem(4, 12, 30, seed=52)
    dp = osvmbe.DeviceProblem.from_host(p)
    ctx = osvmbe.Context()
    with pytest.raises(osvmbe.OsvError) as ei:
        ctx.clusters_build(dp, Params(n_osv_fixed=4, precision=osvmbe.OSV_MIXED_TF32X3))
    assert ei.value.status == osvmbe.OSV_ERR_INVALID
    ctx.close()


@pytest.mark.slow
def test_bf16x4_bench_workload(osvmbe):
    p, prm = workload(1)
    f = run(osvmbe, p, prm)
    prm.precision = 2
    x = run(osvmbe, p, prm)
    dE = x["E"] - f["E"]
    gb = np.abs(x["dB"] - f["dB"]).max()
    gf = np.abs(x["dF"] - f["dF"]).max()
    print(f"\nbench workload mixed vs fp64: E = {f['E']:.9f}, dE = {dE:.3e} Eh (rel {dE / abs(f['E']):.2e}), "
          f"max|d dB| = {gb:.3e} (max|dB| {np.abs(f['dB']).max():.3e}), max|d dF| = {gf:.3e}")
    assert abs(dE) <= 1e-6
    assert gb <= 1e-6 and gf <= 1e-6


@pytest.mark.parametrize("fixed", [0, 7])
def test_mixed_osv_eigenpairs_match_fp64(osvmbe, fixed):
    """FP32 tridiagonal route + FP64 Rayleigh-Ritz refinement: the n_max leading eigenvalues of every T_kk and
    the OSV counts equal the FP64 route's to the accuracy of the mixed T_kk itself (its Gram products come from
    the exact-slice BF16x4 GEMM: ~2^-31 relative per entry, hence ~1e-9 of the largest eigenvalue); the
    remaining eigenvalues are FP32-accurate."""
    p = make_problem(8, 120, 300, seed=61)
    prm = dict(n_osv_max=20, n_osv_fixed=fixed, l_osv=3e-3, mbe_order=3, r2b=6.0, r3b=5.0)
    out = {}
    for prec in (0, 2):
        dp = osvmbe.DeviceProblem.from_host(p)
        ctx = osvmbe.Context()
        ctx.clusters_build(dp, Params(**prm, precision=prec))
        counts = ctx.osv_build(dp, Params(**prm, precision=prec), want_counts=True)
        out[prec] = (counts, np.array([ctx.eigenvalues(k, p.n_vir) for k in range(p.n_occ)]))
        ctx.close()
    nm = fixed if fixed else 20
    assert (out[0][0] == out[2][0]).all()
    w64, wmx = out[0][1], out[2][1]
    scale = np.abs(w64).max()
    lead = np.abs(wmx[:, :nm] - w64[:, :nm]).max() / scale
    rest = np.abs(wmx[:, nm:] - w64[:, nm:]).max() / scale
    print(f"\nleading eigenvalues rel diff {lead:.2e}; rest {rest:.2e}; counts {out[0][0]}")
    assert lead <= 2e-9
    assert rest <= 1e-5


@pytest.mark.parametrize("variant", list(range(13)))
@pytest.mark.parametrize("shape", [(8, 120, 300, 61), (5, 37, 90, 62), (3, 5, 20, 63)])
def test_every_tridiagonalisation_launch_shape(osvmbe, variant, shape):
    """Each launch shape of the FP32 Householder reduction (a pair of CTAs, one CTA with two per SM, clusters of 4, 8
    and 16 CTAs per matrix, one CTA with the updates of two or four steps written together, with or without row
    chunks staged through shared memory), fixed with osv_set_tridiag_variant: the eigenvalues of every T_kk against the FP64
    route, leading ones after the FP64 refinement, the rest straight from the FP32 tridiagonal.  Shapes: rows a
    multiple of four (16-byte passes), an odd order (column-by-column passes), and an order below the cluster
    size (CTAs that own no row)."""
    n_occ, n_vir, n_aux, seed = shape
    p = make_problem(n_occ, n_vir, n_aux, seed=seed)
    nm = min(6, n_vir)
    prm = dict(n_osv_fixed=nm, mbe_order=2, r2b=6.0)
    out = {}
    for prec in (0, 2):
        dp = osvmbe.DeviceProblem.from_host(p)
        ctx = osvmbe.Context()
        if prec:
            ctx.set_tridiag_variant(variant)
        ctx.clusters_build(dp, Params(**prm, precision=prec))
        try:
            ctx.osv_build(dp, Params(**prm, precision=prec), want_counts=True)
        except osvmbe.OsvError as err:   # a cluster size this GPU cannot hold is refused before any launch
            ctx.close()
            if prec and variant == 4 and err.status == osvmbe.OSV_ERR_CUDA and "not supported" in str(err):
                pytest.skip("this GPU holds no cluster of 16 CTAs of this kernel")
            raise
        out[prec] = np.array([ctx.eigenvalues(k, p.n_vir) for k in range(p.n_occ)])
        if prec:
            assert ctx.autotune_report().get("tridiag", {}).get("choice") == "fixed"
        ctx.close()
    scale = np.abs(out[0]).max()
    lead = np.abs(out[2][:, :nm] - out[0][:, :nm]).max() / scale
    rest = np.abs(out[2][:, nm:] - out[0][:, nm:]).max() / scale if n_vir > nm else 0.0
    print(f"\nvariant {variant}, n_vir {n_vir}: leading rel diff {lead:.2e}; rest {rest:.2e}")
    assert lead <= 2e-9 and rest <= 1e-5


@pytest.mark.parametrize("nosv", [6, 41])
def test_bf16x4_adjoint_kernels_match_fp64(osvmbe, nosv):
    """The mixed cluster partials take the tensor-core kernel for pair orders <= 80 (6 OSVs per LMO: orders <= 12)
    and the double-float kernel above (41 OSVs: orders 82); both must give the FP64 path's gradient to the
    mixed path's bar."""
    p = make_problem(5, 60, 200, seed=71)
    base = dict(n_osv_fixed=nosv, mbe_order=3, r2b=6.0, r3b=5.0, tol=1e-11)
    f = run(osvmbe, p, Params(**base))
    x = run(osvmbe, p, Params(**base, precision=2))
    gb = np.abs(x["dB"] - f["dB"]).max()
    gf = np.abs(x["dF"] - f["dF"]).max()
    print(f"\nn_osv {nosv}: dE = {x['E'] - f['E']:.3e}; max|d dB| = {gb:.3e}; max|d dF| = {gf:.3e}")
    assert abs(x["E"] - f["E"]) <= 1e-6
    assert gb <= 1e-6 and gf <= 1e-6


def test_autotuner_reports_its_choices_and_keeps_the_results(osvmbe):
    """The plan-time autotuner times the candidate launch shapes (FP32 tridiagonalisation, double-float GEMM tiles)
    and keeps the fastest; its report names the fixed rule's choice, the tuned one and the timings.  Launch shapes
    change only the rounding order, so the energy with and without tuning agrees to far below the 1e-6 bar."""
    p = make_problem(6, 40, 150, seed=52)
    prm = Params(n_osv_fixed=6, mbe_order=3, r2b=6.0, r3b=5.0, tol=1e-11, precision=2)
    out = {}
    for on in (True, False):
        dp = osvmbe.DeviceProblem.from_host(p)
        ctx = osvmbe.Context()
        ctx.autotune(on)
        ctx.clusters_build(dp, prm)
        out[on] = (osvmbe.run_energy(ctx, dp, prm)[0], ctx.autotune_report())
        ctx.close()
    (E_on, rep), (E_off, rep_off) = out[True], out[False]
    assert rep_off == {}
    tri = rep["tridiag"]
    names = ["cta_pair", "single_cta_2_per_sm", "cluster_4", "cluster_8", "cluster_16", "delayed_2",
             "delayed_2_2_per_sm", "delayed_4", "staged_2_2_per_sm", "staged_2", "staged_2_depth_2",
             "staged_2_depth_3", "staged_2_8_rows"]
    assert set(tri["ms"]) == set(names) and tri["choice"] in names
    timed = {k: v for k, v in tri["ms"].items() if v is not None}   # a cluster size the GPU cannot hold is null
    assert set(names) - {"cluster_16"} <= set(timed)
    whole = tri.get("ms_whole_batch")   # batches above 304 matrices: the two fastest re-timed on the whole batch
    assert (min(whole, key=whole.get) if whole else min(timed, key=timed.get)) == tri["choice"]
    shapes = {"64x64", "80x80", "48x80", "80x48", "48x48"}
    assert rep["gemm_df"] and all(v["rule"] in shapes and v["choice"] in shapes and len(v["ms"]) == 5
                                  for v in rep["gemm_df"].values())
    for v in rep["gemm_df"].values():   # the choice is the fastest timed shape
        assert min(v["ms"]) == v["ms"][["64x64", "80x80", "48x80", "80x48", "48x48"].index(v["choice"])]
    print(f"\nautotuner: {rep}")
    assert abs(E_on - E_off) <= 1e-9
