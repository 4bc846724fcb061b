"""The derivative kernels of the progressive use case (Sec. 5.3) against the
oracle, bit for bit (both sides compute in the field's type, one rounding per
operation in one order): ragged 3D, 2D and 1D fields, every axis, spacings
whose 2h or h^2 is a power of two (multiplication by the reciprocal) and
others (division), the smallest extents the stencils allow, and the argument
checks.  Then the use case itself: on progressive reconstructions of a
velocity field the derivatives' errors stay within the bounds that the
stencils and Eq. 1 give (|d omega| <= 8 tau / h, |d w_zz| <= 12 tau / h^2),
and shrink with k."""
import numpy as np
import pytest

import synth_fields as S
from oracle import derivatives as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    import paper_2308_11759_gb300 as pcz

    pcz.lib()
    return pcz


def _bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


# rows that are a multiple of 4 values long take the float32 vector kernel
SHAPES = [(37, 29, 45), (9, 130, 7), (3, 3, 3), (4, 5, 4), (50, 33), (3, 3), (13, 20, 132), (5, 3, 4), (7, 11, 260)]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("h", [1.0, 0.5, 0.1, 3.0])
def test_vorticity_equals_oracle(P, dtype, h):
    for j, shape in enumerate(SHAPES):
        u = S.powerlaw(shape, seed=300 + j, dtype=dtype)
        v = S.powerlaw(shape, seed=400 + j, dtype=dtype)
        got = P.fd_vorticity_z(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), h).cpu().numpy()
        assert np.array_equal(_bits(got), _bits(D.vorticity_z(u, v, h))), shape


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("h", [1.0, 0.25, 0.3])
def test_second_derivative_equals_oracle(P, dtype, h):
    cases = [((37, 29, 45), (0, 1, 2)), ((4, 6, 300), (0, 1, 2)), ((50, 33), (0, 1)), ((1001,), (0,)), ((4,), (0,))]
    for j, (shape, axes) in enumerate(cases):
        w = S.powerlaw(shape, seed=500 + j, dtype=dtype) if len(shape) > 1 else \
            np.random.default_rng(j).standard_normal(shape).astype(dtype)
        wd = torch.from_numpy(w).cuda()
        for axis in axes:
            if shape[len(shape) - 1 - axis] < 4:
                continue
            got = P.fd_second(wd, axis, h).cpu().numpy()
            assert np.array_equal(_bits(got), _bits(D.second(w, axis, h))), (shape, axis)


def test_vector_and_scalar_vorticity_agree(P):
    # the same float32 field through the vector kernel (16-byte aligned) and
    # through the scalar one (arrays starting 4 bytes off alignment)
    u = S.powerlaw((11, 17, 136), seed=900, dtype=np.float32)
    v = S.powerlaw((11, 17, 136), seed=901, dtype=np.float32)
    a = P.fd_vorticity_z(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), 0.5)
    n = u.size
    bu, bv, bo = (torch.empty(n + 1, device="cuda") for _ in range(3))
    uo, vo, oo = bu[1:].view(u.shape), bv[1:].view(u.shape), bo[1:].view(u.shape)
    uo.copy_(torch.from_numpy(u))
    vo.copy_(torch.from_numpy(v))
    P.fd_vorticity_z(uo, vo, 0.5, out=oo)
    assert uo.data_ptr() % 16 != 0
    assert torch.equal(a.view(torch.int32), oo.view(torch.int32))
    assert np.array_equal(_bits(a.cpu().numpy()), _bits(D.vorticity_z(u, v, 0.5)))


def test_large_field_sampled(P):
    # a 256^3 float32 field in the launch shape of the use-case leg: every
    # boundary face and a random sample of interior points, against the oracle
    u = S.powerlaw((256, 256, 256), seed=7, dtype=np.float32)
    v = S.powerlaw((256, 256, 256), seed=8, dtype=np.float32)
    om = P.fd_vorticity_z(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), 1.0).cpu().numpy()
    ww = P.fd_second(torch.from_numpy(v).cuda(), 2, 1.0).cpu().numpy()
    want_om = D.vorticity_z(u, v, 1.0)
    want_ww = D.second(v, 2, 1.0)
    rng = np.random.default_rng(1)
    idx = tuple(rng.integers(0, 256, size=(3, 20000)))
    for got, want in ((om, want_om), (ww, want_ww)):
        assert np.array_equal(_bits(got[idx]), _bits(want[idx]))
        for face in (np.s_[0], np.s_[-1], np.s_[:, 0], np.s_[:, -1], np.s_[:, :, 0], np.s_[:, :, -1]):
            assert np.array_equal(_bits(got[face]), _bits(want[face]))


def test_argument_checks(P):
    x = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(P.PczError):
        P.fd_second(x, 3)  # axis beyond the field
    with pytest.raises(P.PczError):
        P.fd_second(torch.zeros((3, 8, 8), device="cuda"), 2)  # 3 points along z
    with pytest.raises(P.PczError):
        P.fd_vorticity_z(torch.zeros(8, device="cuda"), torch.zeros(8, device="cuda"))  # 1D
    with pytest.raises(P.PczError):
        P.fd_vorticity_z(torch.zeros((8, 2, 8), device="cuda"), torch.zeros((8, 2, 8), device="cuda"))  # ny = 2
    with pytest.raises(P.PczError):
        P.fd_second(x, 0, h=0.0)
    with pytest.raises(P.PczError):
        P.fd_second(x, 0, h=float("inf"))
    with pytest.raises(P.PczError):
        P.fd_second(x, 0, out=x)  # in place
    with pytest.raises(P.PczError):
        P.fd_second(torch.zeros((8, 8, 8)), 0, out=torch.zeros((8, 8, 8)))  # host memory


def test_use_case_error_bounds(P):
    """Sec. 5.3: a velocity field in 3 components, each compressed with
    tau = 1, 2^-4, 2^-9 (the tolerances the paper uses); at every k the
    derivatives of x~_k stay within the stencil bounds of Eq. 1 and their
    errors fall with k."""
    shape = (64, 72, 80)
    vel = [S.powerlaw(shape, seed=600 + c, dtype=np.float64) * 4.0 for c in range(3)]
    tau = [1.0, 2.0 ** -4, 2.0 ** -9]
    h = 1.0
    dev = [torch.from_numpy(c).cuda() for c in vel]
    streams = [P.compress(c, tau) for c in dev]
    om_ref = P.fd_vorticity_z(dev[0], dev[1], h)
    wzz_ref = P.fd_second(dev[2], 2, h)
    prev = None
    for k in (1, 2, 3):
        rec = [s.retrieve(k=k) for s in streams]
        for c in range(3):
            assert float((rec[c] - dev[c]).abs().max()) <= tau[k - 1]
        d_om = float((P.fd_vorticity_z(rec[0], rec[1], h) - om_ref).abs().max())
        d_wzz = float((P.fd_second(rec[2], 2, h) - wzz_ref).abs().max())
        assert d_om <= 8 * tau[k - 1] / h * (1 + 1e-12)
        assert d_wzz <= 12 * tau[k - 1] / h ** 2 * (1 + 1e-12)
        if prev:
            assert d_om < prev[0] and d_wzz < prev[1]
        prev = (d_om, d_wzz)
    for s in streams:
        s.close()
