"""Entry images (mixed precision, built-in kernel operators): a factorization
that forms every kernel entry once per orientation and feeds all its
structured sketches (Alg. 2, Sec. 4.1) from those images computes the same
bf16 parts and products as one that forms the entries on the fly in every
sketch, summed in another order -- so the two agree to FP32 rounding: the
same ranks (+-1 where a pivot sits at the threshold), applies within 1e-5,
sketch errors within the Thm 5.3 bound.  Cases: chunk-aligned trees (every
sketch reads the images), ragged trees (groups off the 16-column grid fall
back to on-the-fly entries), 3D and DFT kernels, and a memory cap too small
for the images (no images at all: bit-identical)."""
import numpy as np
import pytest
import torch

from paper_2002_03400_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _factor(plan, images):
    api.set_entry_images(images)
    try:
        op = api.Operator.kernel(plan)
        F = api.Factorization.factor(plan, op)
    finally:
        api.set_entry_images(True)
    return F, op


def _close(a, b, tol=1e-5):
    torch.cuda.synchronize()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(a)) <= tol


def _same(plan, n_in, seed=3):
    Fa, op = _factor(plan, False)
    Fb, _ = _factor(plan, True)
    worst = 0
    for side, levels in ((0, range(plan.lm + 1)), (1, range(plan.lm, plan.L + 1))):
        for j in levels:
            worst = max(worst, int(np.max(np.abs(Fa.ranks(side, j) - Fb.ranks(side, j)))))
    assert worst <= 1
    x = api.colmajor(torch.from_numpy(inputs.random_rhs(n_in, 5, seed=seed)).to(torch.complex64).cuda())
    assert _close(Fa.apply(x), Fb.apply(x))
    for opn in ("T", "C"):
        xt = api.colmajor(torch.from_numpy(inputs.random_rhs(plan.m, 3, seed=seed + 1)).to(torch.complex64).cuda())
        assert _close(Fa.apply(xt, opn), Fb.apply(xt, opn))
    return Fa, Fb, op


@pytest.mark.parametrize("n", [2048, 4096])
def test_images_match_line_pair(n):
    g = inputs.line_pair(n)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6,
                    precision="mixed", r0=16)
    Fa, Fb, op = _same(plan, n)
    ea = Fa.error(op, 16, seed=2, dtype=torch.complex64)
    eb = Fb.error(op, 16, seed=2, dtype=torch.complex64)
    bound = 2 * np.sqrt(plan.L + 2) * 1e-6
    assert ea <= bound and eb <= bound and abs(ea - eb) <= 0.05 * bound


@pytest.mark.parametrize("geom,n,m,leaf", [("arc", 1000, 900, 16), ("cap", 777, 700, 24), ("line", 300, 300, 8)])
def test_images_match_ragged(geom, n, m, leaf):
    g = {"arc": lambda: inputs.arc_pair(n, seed=2, m=m), "cap": lambda: inputs.cap_pair(n, m=m),
         "line": lambda: inputs.line_pair(n, m)}[geom]()
    plan = api.Plan(g.src, g.tgt, kernel=g.kernel, wavenumber=g.wavenumber, leaf=leaf, tol=1e-6,
                    precision="mixed")
    _same(plan, n)


def test_images_match_dft():
    n = 1024
    g = inputs.dft_points(n)
    plan = api.Plan(g.src, g.tgt, kernel="dft", leaf=16, tol=1e-6, precision="mixed")
    _same(plan, n)


def test_images_skipped_under_memory_cap():
    n = 2048
    g = inputs.line_pair(n)
    kw = dict(kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6, precision="mixed", r0=16)
    # room for the factorization; the two images (2 x 16.8 MB here) would take
    # more than half of the cap, so they are not formed
    plan = api.Plan(g.src, g.tgt, mem_cap=64 * 1024 * 1024, **kw)
    ref = api.Plan(g.src, g.tgt, **kw)
    F, _ = _factor(plan, True)
    Fr, _ = _factor(ref, False)
    x = api.colmajor(torch.from_numpy(inputs.random_rhs(n, 2, seed=1)).to(torch.complex64).cuda())
    assert torch.equal(F.apply(x), Fr.apply(x))


def test_set_entry_images_rejects_bad_values():
    assert api.lib().bf_set_entry_images(2) == -1
    assert api.lib().bf_set_entry_images(1) == 0


def test_cached_kernel_operator_products_and_factorization():
    """bf_operator_kernel_cached: products with A, A^T, A^H stream the
    resident images and match the FP64 kernel entries to FP32 level; a
    factorization of the cached operator reuses them and matches one of the
    plain operator."""
    from oracle import operators as oo
    n = 1536
    g = inputs.line_pair(n)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6,
                    precision="mixed", r0=16)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    opc = api.Operator.kernel(plan, cached=True)
    x = inputs.random_rhs(n, 7, seed=2)
    xt = torch.from_numpy(x).to(torch.complex64).cuda()
    for opn, ref in (("N", A @ x), ("T", A.T @ x), ("C", A.conj().T @ x)):
        y = opc.apply(api.colmajor(xt), opn)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - ref) <= 2e-6 * np.linalg.norm(ref)
    Fc = api.Factorization.factor(plan, opc)
    Fp, _ = _factor(plan, True)
    xr = api.colmajor(torch.from_numpy(inputs.random_rhs(n, 3, seed=5)).to(torch.complex64).cuda())
    assert _close(Fc.apply(xr), Fp.apply(xr))
    assert Fc.error(opc, 16, seed=3, dtype=torch.complex64) <= 2 * np.sqrt(plan.L + 2) * 1e-6


def test_repeated_factorizations_stay_within_bound():
    """Eight factorizations of the n = 16384 workload (entry images, the
    warp-specialized sketch kernel's pipeline under varying timing): every
    sketch error stays within the Thm 5.3 bound and the ranks repeat."""
    n = 16384
    g = inputs.line_pair(n)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6,
                    precision="mixed", r0=16)
    op = api.Operator.kernel(plan)
    bound = 2 * np.sqrt(plan.L + 2) * 1e-6
    first = None
    for _ in range(8):
        F = api.Factorization.factor(plan, op)
        assert F.error(op, 16, seed=3, dtype=torch.complex64) <= bound
        r = np.concatenate([F.ranks(0, j) for j in range(plan.lm + 1)])
        if first is None:
            first = r
        assert np.array_equal(r, first)


@pytest.mark.parametrize("ncols", [3, 12, 20, 30])
def test_cached_products_every_tile_width(ncols):
    """Products of the cached operator at every tile width of the image
    kernel (NR = 16, 32, 48 real columns with the A parts in tensor memory,
    64 with them in shared memory), on a ragged grid (1000 rows: seven full
    128-row tiles and a tail of 104; 1300 columns: a tail of 4 past the last
    16-column chunk), against the FP64 kernel entries of the oracle: every
    orientation within FP32 level."""
    from oracle import operators as oo
    n, m = 1300, 1000
    g = inputs.line_pair(n, m)
    plan = api.Plan(g.src, g.tgt, kernel="helmholtz2d", wavenumber=g.wavenumber, leaf=16, tol=1e-6,
                    precision="mixed", r0=16)
    A = oo.kernel_entries(oo.HELMHOLTZ_2D, g.wavenumber, g.tgt, g.src)
    opc = api.Operator.kernel(plan, cached=True)
    for opn, rows, ref_of in (("N", n, lambda x: A @ x), ("T", m, lambda x: A.T @ x), ("C", m, lambda x: A.conj().T @ x)):
        x = inputs.random_rhs(rows, ncols, seed=ncols)
        y = opc.apply(api.colmajor(torch.from_numpy(x).to(torch.complex64).cuda()), opn)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.complex128)
        ref = ref_of(x.astype(np.complex64).astype(np.complex128))
        assert got.shape == ref.shape
        assert np.linalg.norm(got - ref) <= 2e-6 * np.linalg.norm(ref), opn
