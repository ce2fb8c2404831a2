"""Shared helpers for the test-suite: cached meshes, oracle results and the
FP64-contract tolerances (|dn| <= 1e-12 h^(D-1), |dV| <= 1e-12 h^D,
|dbnormal| <= 1e-12 h^(D-1), |dgrad| <= 1e-12 max|grad|)."""
import functools

import numpy as np

import meshgen
import oracle

TOL_N = 1e-12
TOL_V = 1e-12
TOL_G = 1e-12

SMALL_MESHES = {
    "tri16": lambda: meshgen.workload("tri16"),
    "tri_odd": lambda: meshgen.tri_square(13, jitter=0.3, seed=501),
    "single2": lambda: meshgen.single_simplex(2, seed=502),
    "single3": lambda: meshgen.single_simplex(3, seed=503),
    "kuhn5": lambda: meshgen.kuhn_cube(5, jitter=0.3, seed=504),
    "kuhn7_off": lambda: meshgen.kuhn_cube(7, jitter=0.25, seed=505, offset=1000.0),
    "kuhn11_nomorton": lambda: meshgen.kuhn_cube(11, jitter=0.2, seed=506, morton=False),
    "kuhn48": lambda: meshgen.workload("kuhn48"),
}


@functools.lru_cache(maxsize=None)
def mesh(name):
    return SMALL_MESHES[name]()


@functools.lru_cache(maxsize=None)
def oracle_topo(name):
    m = mesh(name)
    return oracle.topology(m.dim, m.elems, m.x)


@functools.lru_cache(maxsize=None)
def oracle_fwd(name):
    m = mesh(name)
    return oracle.direct(m.dim, m.x, m.elems, oracle_topo(name))


@functools.lru_cache(maxsize=None)
def loss_weights(name):
    m = mesh(name)
    t = oracle_topo(name)
    return meshgen.generate.loss_weights(t.n_edges, m.n_nodes, m.dim, seed=meshgen.SEED_BASE + 5)


def hscale(m):
    return m.h if m.n_elems > 1 else 1.0


def assert_close_n(got, ref, m, what="n"):
    tol = TOL_N * hscale(m) ** (m.dim - 1)
    err = np.abs(np.asarray(got) - np.asarray(ref)).max() if np.size(ref) else 0.0
    assert err <= tol, f"{what}: max |diff| {err:.3e} > {tol:.3e}"
    return err


def assert_close_v(got, ref, m):
    tol = TOL_V * hscale(m) ** m.dim
    err = np.abs(np.asarray(got) - np.asarray(ref)).max()
    assert err <= tol, f"V: max |diff| {err:.3e} > {tol:.3e}"
    return err


def assert_close_g(got, ref):
    ref = np.asarray(ref)
    tol = TOL_G * np.abs(ref).max()
    err = np.abs(np.asarray(got) - ref).max()
    assert err <= tol, f"grad: max |diff| {err:.3e} > {tol:.3e}"
    return err
