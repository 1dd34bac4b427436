"""CPU-only checks of the C ABI: the library builds, loads, exports every symbol
declared in include/hz.h, and its host-side analysis (hz_plan) agrees with the
oracle's dof counts and decomposition sizes.  No device call is made."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import dd, fem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hzmod():
    from paper_2004_06309_gb300 import build, hz
    build.build()
    return hz


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hz_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(hzmod):
    lib = hzmod.load()
    names = declared_symbols()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
        assert name in hzmod.SIGNATURES, name


def test_status_strings(hzmod):
    lib = hzmod.lib()
    assert lib.hz_status_string(0) == b"ok"
    assert lib.hz_status_string(5) == b"zero pivot"


@pytest.mark.parametrize("make", [
    lambda: synth.tiny_problem(),
    lambda: synth.unit_cube_problem(n=6, order=2, nsub=4, overlap=2),
    lambda: synth.small_overthrust(levels=2, cells=(3, 3, 2), freq=0.8, nsub=4),
])
def test_plan_matches_oracle_sizes(hzmod, make):
    p = make()
    st = hzmod.plan(p)
    A, dm, dd_ = fem.global_system(p)
    assert st["n"] == dm.n
    subs = dd.grow_subdomains(p.mesh, p.elem_part, p.nsub, p.overlap, dm)
    assert st["sum_ni"] == sum(len(s.dofs) for s in subs)
    # nnz of A counts the element pattern (explicit zeros kept on Dirichlet couplings)
    assert st["nnz"] >= A.nnz
    assert st["nnz_factor"] > 0 and st["nsupernodes"] > 0
    if p.levels == 2:
        from oracle import coarse
        Z, cdm, keep = coarse.interpolation(p, dm)
        assert st["n_coarse"] == Z.shape[1]


def test_plan_rejects_bad_options(hzmod):
    bad = synth.tiny_problem()
    bad.restart = 0
    with pytest.raises(hzmod.HzError):
        hzmod.plan(bad)
    p2 = synth.tiny_problem()
    p2.levels = 2          # no coarse mesh given
    with pytest.raises(hzmod.HzError):
        hzmod.plan(p2)


def test_plan_builtin_partition(hzmod):
    p = synth.tiny_problem()
    a = hzmod.plan(p, use_partition=True)
    b = hzmod.plan(p, use_partition=False)   # the library's own coordinate bisection
    assert a["sum_ni"] == b["sum_ni"]


def test_sweep_schedules_cover_every_kernel_variant(hzmod):
    """The case test_gpu_variants runs on the GPU: across the default, wide-everywhere and
    narrow-everywhere schedules (host-only analysis) every sweep variant occurs, with
    128-wide complex64 supernodes (112 in FP64), split backward column blocks and
    multi-tile, multi-stage tensor-core Schur updates; bad schedule options are rejected."""
    p = synth.overthrust_problem(seed=0, freq=1.25, nsub=7, overlap=2, restart=50, levels=2)
    for prec, width in ((hzmod.HZ_FP64, 112), (hzmod.HZ_MIXED, 128)):
        plans = {sw: hzmod.plan(p, precision=prec, sweep_tasks=sw) for sw in (0, 1, 2)}
        for st in plans.values():
            assert st["max_snode_width"] == width
            assert st["fwd_levels_wide"] + st["fwd_levels_narrow"] == st["solve_levels"]
            assert st["bwd_levels_wide"] + st["bwd_levels_narrow"] == st["solve_levels"]
            assert st["bwd_split_blocks"] > 0
        assert plans[1]["fwd_levels_narrow"] == 0 and plans[1]["bwd_levels_narrow"] == 0
        assert plans[2]["fwd_levels_wide"] == 0 and plans[2]["bwd_levels_wide"] == 0
        if prec == hzmod.HZ_MIXED:
            st = plans[0]
            assert st["tc_multi_fronts"] > 0 and st["tc_max_kstages"] == 8
            assert st["tc_tiles"] > st["tc_multi_fronts"]
    for bad in (dict(sweep_tasks=3), dict(bwd_chunk=31), dict(bwd_chunk=33), dict(bwd_chunk=514)):
        with pytest.raises(hzmod.HzError):
            hzmod.plan(synth.tiny_problem(), **bad)


def test_factor_groups_shrink_the_frontal_workspace(hzmod):
    """Factorising the subdomains in groups plans each group's fronts from the start of one
    workspace: the workspace shrinks, nothing else in the plan changes."""
    p = synth.overthrust_problem(seed=0, freq=1.25, nsub=8, overlap=2, restart=50, levels=2)
    a = hzmod.plan(p, precision=hzmod.HZ_MIXED)
    b = hzmod.plan(p, precision=hzmod.HZ_MIXED, factor_group=2)
    assert b["front_bytes"] < a["front_bytes"]
    for key in ("n", "sum_ni", "nnz_factor", "nnz_local", "nsupernodes", "device_bytes"):
        assert a[key] == b[key], key
    with pytest.raises(hzmod.HzError):
        hzmod.plan(p, factor_group=-1)


@pytest.mark.parametrize("n", [1, 2, 3, 8, 33, 66])
def test_dense_eig_against_known_spectra(hzmod, n):
    """The host eigen-solver of the GCRO-DR cycle end (Hessenberg reduction, shifted QR,
    back substitution): eigenpairs satisfy A v = w v to rounding and match numpy's
    eigenvalues; a matrix built as Q T Q^H returns the diagonal of T."""
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    w, V = hzmod.dense_eig(A)
    assert np.linalg.norm(A @ V - V * w) <= 1e-13 * np.linalg.norm(A) * max(1, n)
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0)
    ref = np.linalg.eigvals(A)
    assert max(np.min(np.abs(x - ref)) for x in w) <= 1e-11 * np.abs(ref).max()
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    lam = np.arange(1, n + 1) * (1 + 0.5j)
    T = np.triu(rng.standard_normal((n, n)), 1) + np.diag(lam)
    w2, V2 = hzmod.dense_eig(Q @ T @ Q.conj().T)
    assert np.allclose(np.sort_complex(w2), np.sort_complex(lam), atol=1e-10 * n)


def test_dense_eig_real_pairs_diagonal_and_bad_input(hzmod):
    rng = np.random.default_rng(4)
    R = rng.standard_normal((20, 20))                 # real: conjugate eigenvalue pairs
    w, V = hzmod.dense_eig(R)
    assert np.linalg.norm(R @ V - V * w) <= 1e-13 * np.linalg.norm(R) * 20
    D = np.diag(np.arange(1.0, 7.0))                  # already triangular: deflates at once
    w, V = hzmod.dense_eig(D)
    assert np.allclose(np.sort(w.real), np.arange(1.0, 7.0)) and np.allclose(w.imag, 0)
    bad = np.full((3, 3), np.nan + 0j)
    with pytest.raises(hzmod.HzError) as e:
        hzmod.dense_eig(bad)
    assert e.value.status == hzmod.HZ_ERR_BREAKDOWN


def test_solve_trees_merge_the_separator_chains(hzmod):
    """The direct coarse factor's sweeps run on a solve tree with the supernode chains at the
    top separators merged: fewer levels than the factor tree, merged widths within 448; the
    subdomain factors' sweeps likewise on their sparse top levels; the iterative coarse
    solve has no direct factor and merges nothing there."""
    import bench
    p = bench.make_problem(bench.WORKLOADS["overthrust-small"])
    st = hzmod.plan(p, precision=hzmod.HZ_MIXED)
    assert st["coarse_merged_chains"] > 0
    assert 0 < st["coarse_solve_levels"] < st["nlevels_coarse"], st
    # a merged chain's panel holds at most 448 columns of n_coarse rows
    assert 0 < st["coarse_merged_bytes"] <= st["coarse_merged_chains"] * 448 * st["n_coarse"] * 16
    # the subdomain factors: chains merge on the sparse top levels only
    assert st["merged_chains"] > 0 and 0 < st["solve_levels"] < st["nlevels"], st
    assert 0 < st["merged_bytes"] < st["nnz_factor"] * 8
    it = hzmod.plan(p, precision=hzmod.HZ_MIXED, coarse_solver=hzmod.HZ_COARSE_ORAS)
    assert it["coarse_merged_chains"] == 0 and it["coarse_merged_bytes"] == 0
    assert it["coarse_solve_levels"] == it["nlevels_coarse"]


def test_solve_tree_merge_off_plans_the_factor_trees(hzmod):
    """With HZ_NO_SOLVE_MERGE set (read once per process, hence a child process) the
    sweeps are planned on the factor trees: as many solve levels as factor levels, no
    merged panels, and planned device bytes lower by the merged panels' bytes plus the 5 %
    headroom the plan adds to everything it counts."""
    import json
    import subprocess
    import sys
    code = ("import json, bench\n"
            "from paper_2004_06309_gb300 import hz\n"
            "p = bench.make_problem(bench.WORKLOADS['overthrust-small'])\n"
            "out = {}\n"
            "for prec in (hz.HZ_MIXED, hz.HZ_FP64):\n"
            "    out[prec] = hz.plan(p, precision=prec)\n"
            "print(json.dumps(out))\n")
    runs = {}
    for off in (False, True):
        env = dict(os.environ)
        env.pop("HZ_NO_SOLVE_MERGE", None)
        if off:
            env["HZ_NO_SOLVE_MERGE"] = "1"
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        runs[off] = json.loads(r.stdout.strip().splitlines()[-1])
    for prec in runs[False]:
        on, off = runs[False][prec], runs[True][prec]
        assert off["solve_levels"] == off["nlevels"] and off["coarse_solve_levels"] == off["nlevels_coarse"]
        assert off["merged_chains"] == 0 and off["merged_bytes"] == 0
        assert off["coarse_merged_chains"] == 0 and off["coarse_merged_bytes"] == 0
        assert on["merged_bytes"] > 0 and on["coarse_merged_bytes"] > 0
        assert on["nnz_factor"] == off["nnz_factor"] and on["nlevels"] == off["nlevels"]
        merged = on["merged_bytes"] + on["coarse_merged_bytes"]
        assert abs(on["device_bytes"] - off["device_bytes"] - 1.05 * merged) <= 2, (on, off)
