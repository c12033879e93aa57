"""Pins of the oracle's resolution change (oracle.topopt.resample: the design
interpolation of Sec. 3 / Sec. 4.1 between grids) against what the
definitions fix independently of its index formulas:

* kind 0 (piecewise constant): a brute-force loop over fine elements; the mean
  is preserved exactly;
* kind 1 (trilinear between cell centres): pointwise evaluation in physical
  coordinates by a plain loop; constants kept, values stay in the input's
  range, linear fields reproduced between the outermost centres;
* kind 2 (nodal Q1 embedding): the coarse trilinear shape functions evaluated
  at the fine nodes' physical coordinates by a plain loop; and, because the
  fine field is the same function, its integral f^T u and its energy
  u^T A u (conductivity carried by kind 0) equal the coarse ones.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, topopt

CASES = [((3, 2, 4), (6, 4, 8)), ((2, 3, 2), (2, 6, 8)), ((4, 4, 4), (4, 4, 4))]


@pytest.mark.parametrize("gc,gf", CASES)
def test_piecewise_constant_by_brute_force(gc, gf):
    Mc = gc[0] * gc[1] * gc[2]
    v = W.uniform01(71, Mc)
    out = topopt.resample(gc, v, gf, 0)
    r = [f // c for f, c in zip(gf, gc)]
    for e in range(gf[0] * gf[1] * gf[2]):
        ix, iy, iz = e % gf[0], (e // gf[0]) % gf[1], e // (gf[0] * gf[1])
        ec = ix // r[0] + gc[0] * (iy // r[1] + gc[1] * (iz // r[2]))
        assert out[e] == v[ec]
    assert abs(out.mean() - v.mean()) <= 1e-15


def _lin1(cc, x):
    """Linear interpolation of samples at sorted points cc, constant outside."""
    if x <= cc[0]:
        return 0, 0, 0.0
    if x >= cc[-1]:
        return len(cc) - 1, len(cc) - 1, 0.0
    k = int(np.searchsorted(cc, x, side="right")) - 1
    return k, k + 1, (x - cc[k]) / (cc[k + 1] - cc[k])


@pytest.mark.parametrize("gc,gf", CASES)
def test_cell_trilinear_pointwise(gc, gf):
    Mc = gc[0] * gc[1] * gc[2]
    v = W.uniform01(72, Mc)
    out = topopt.resample(gc, v, gf, 1)
    # physical coordinates on the unit box: centres of coarse cells, of fine cells
    cen = [(np.arange(gc[k]) + 0.5) / gc[k] for k in range(3)]
    for e in range(gf[0] * gf[1] * gf[2]):
        idx = (e % gf[0], (e // gf[0]) % gf[1], e // (gf[0] * gf[1]))
        w = [_lin1(cen[k], (idx[k] + 0.5) / gf[k]) for k in range(3)]
        s = 0.0
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    wt = ((w[0][2] if cx else 1 - w[0][2]) * (w[1][2] if cy else 1 - w[1][2])
                          * (w[2][2] if cz else 1 - w[2][2]))
                    i = w[0][1] if cx else w[0][0]
                    j = w[1][1] if cy else w[1][0]
                    k = w[2][1] if cz else w[2][0]
                    s += wt * v[i + gc[0] * (j + gc[1] * k)]
        assert abs(out[e] - s) <= 1e-15, (e, out[e], s)
    assert out.min() >= v.min() - 1e-15 and out.max() <= v.max() + 1e-15
    np.testing.assert_array_equal(topopt.resample(gc, np.full(Mc, 0.3), gf, 1), np.full(out.size, 0.3))


def test_cell_trilinear_reproduces_linear_fields_inside():
    gc, gf = (4, 4, 4), (8, 8, 8)
    cen = (np.arange(4) + 0.5) / 4
    ez, ey, ex = np.meshgrid(cen, cen, cen, indexing="ij")
    v = (1.0 + 2.0 * ex - 3.0 * ey + 0.5 * ez).ravel()
    out = topopt.resample(gc, v, gf, 1).reshape(8, 8, 8)
    cf = (np.arange(8) + 0.5) / 8
    fz, fy, fx = np.meshgrid(cf, cf, cf, indexing="ij")
    ref = 1.0 + 2.0 * fx - 3.0 * fy + 0.5 * fz
    inside = (slice(1, 7),) * 3  # fine centres between the outermost coarse centres
    np.testing.assert_allclose(out[inside], ref[inside], rtol=0, atol=1e-14)


@pytest.mark.parametrize("gc,gf", CASES)
def test_nodal_embedding_pointwise(gc, gf):
    nc = fem.n_nodes(gc)
    u = W.uniform01(73, nc) - 0.5
    out = topopt.resample(gc, u, gf, 2)
    nxf, nyf = gf[0] + 1, gf[1] + 1
    for n in range(fem.n_nodes(gf)):
        p = (n % nxf / gf[0], (n // nxf) % nyf / gf[1], n // (nxf * nyf) / gf[2])
        # containing coarse element (the last one on the upper faces) and local coordinates
        e = [min(int(np.floor(p[k] * gc[k])), gc[k] - 1) for k in range(3)]
        loc = [p[k] * gc[k] - e[k] for k in range(3)]
        s = 0.0
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, a >> 2
            phi = ((loc[0] if ax else 1 - loc[0]) * (loc[1] if ay else 1 - loc[1]) * (loc[2] if az else 1 - loc[2]))
            s += phi * u[(e[0] + ax) + (gc[0] + 1) * ((e[1] + ay) + (gc[1] + 1) * (e[2] + az))]
        assert abs(out[n] - s) <= 1e-15, (n, out[n], s)


@pytest.mark.parametrize("gc,gf", CASES[:2])
def test_nodal_embedding_keeps_integral_and_energy(gc, gf):
    hc = tuple(1.0 / g for g in gc)
    hf = tuple(1.0 / g for g in gf)
    Mc = gc[0] * gc[1] * gc[2]
    u = W.uniform01(74, fem.n_nodes(gc)) - 0.5
    uf = topopt.resample(gc, u, gf, 2)
    fc = fem.load_vector(gc, hc, np.ones(Mc))
    ff = fem.load_vector(gf, hf, np.ones(gf[0] * gf[1] * gf[2]))
    assert abs(ff @ uf - fc @ u) <= 1e-14 * np.abs(fc) @ np.abs(u)
    kc = 1e-3 + W.uniform01(75, Mc)
    kf = topopt.resample(gc, kc, gf, 0)
    Ec = u @ (fem.assemble_neumann(gc, hc, kc) @ u)
    Ef = uf @ (fem.assemble_neumann(gf, hf, kf) @ uf)
    assert abs(Ef - Ec) <= 1e-12 * abs(Ec), (Ef, Ec)


def test_rejects_non_integer_ratios():
    with pytest.raises(ValueError):
        topopt.resample((4, 4, 4), np.zeros(64), (6, 8, 8), 0)
    with pytest.raises(ValueError):
        topopt.resample((4, 4, 4), np.zeros(64), (8, 8, 8), 3)
