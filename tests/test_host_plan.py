"""The context's allocation plan (thermo_plan_bytes: thermo_create's
allocation code run without allocating) on the CPU: the lean FP32-only
hierarchy is smaller than the default form, which is smaller than the FP64
form; a Dirichlet-value array adds exactly one padded FP64 node vector; the
plan grows with the element count; options thermo_create rejects are
rejected here too.  The same plan is checked against the device memory a
real context takes in tests/test_gpu_lean.py."""
import pytest

from paper_2410_06850_gb300 import build, thermo as T


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _nsize(N):
    # padded node vector of the layout: base 32 + (nz + 2) rows of (Ny + 3) x P, + 64
    P = ((N + 3 + 31) // 32) * 32
    return 32 + (N + 3) * (N + 3) * P + 64


def test_forms_are_ordered():
    for N in (32, 64, 128):
        g = (N, N, N)
        lean = T.plan_bytes(g, lean=1, density_fp32=1)
        mixed = T.plan_bytes(g)
        fp64 = T.plan_bytes(g, prec=0)
        assert 0 < lean < mixed < fp64, (N, lean, mixed, fp64)


def test_dirichlet_values_add_one_vector():
    for N in (32, 64):
        g = (N, N, N)
        d = T.plan_bytes(g, has_dirichlet_value=True) - T.plan_bytes(g)
        assert d == (_nsize(N) * 8 + 64 + 511) // 512 * 512


def test_fp32_design_halves_the_design_copy():
    N = 64
    d = T.plan_bytes((N,) * 3) - T.plan_bytes((N,) * 3, density_fp32=1)
    M = N ** 3
    assert d == (M * 8 + 64 + 511) // 512 * 512 - (M * 4 + 64 + 511) // 512 * 512


def test_plan_scales_with_the_grid():
    # 512^3 and 1024^3 share the 8,704-unknown coarsest level (three dense n x n FP64
    # arrays, 1.8 GB): the rest grows with the element count
    a = T.plan_bytes((512,) * 3, lean=1, density_fp32=1)
    big = T.plan_bytes((1024,) * 3, lean=1, density_fp32=1)
    dense = 3 * 8704 ** 2 * 8
    assert 7.5 < (big - dense) / (a - dense) < 8.2
    # the 1024^3 context: FP32 hierarchy, FP64 outer vectors; well inside one GPU's HBM
    assert 150e9 < big < 200e9, big / 1e9


def test_rejections():
    with pytest.raises(T.ThermoError):
        T.plan_bytes((64, 64, 64), lean=1, prec=0)  # lean needs a mixed form
    with pytest.raises(T.ThermoError):
        T.plan_bytes((64, 64, 64), lean=1, pc=1)  # and the MMG preconditioner
    with pytest.raises(T.ThermoError):
        T.plan_bytes((64, 64, 66))  # not a multiple of the block
    with pytest.raises(T.ThermoError):
        T.plan_bytes((64, 64, 64), lean=2)
