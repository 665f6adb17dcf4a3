"""gp_call_bytes without a GPU: the device memory each call would take, from
host arithmetic alone (default options, no budget).  Checked against what the
calls must hold (the packed tiles of R per candidate, the model's copy of x),
the affine growth with the batch, and the argument errors."""
import pytest

pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gp():
    from paper_1203_1269_gb300 import build
    build.build()
    from paper_1203_1269_gb300 import gp as gp_mod
    return gp_mod


def packed_bytes(n):
    nt = (n + 127) // 128
    return nt * (nt + 1) // 2 * 128 * 128 * 8


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_batch_workspace_is_affine_in_T(gp, prec):
    b = {T: gp.call_bytes("nll_batch", 1000, 6, T, prec) for T in (1, 2, 9, 256)}
    per = b[2] - b[1]
    assert b[9] - b[1] == 8 * per and b[256] - b[1] == 255 * per
    assert 0 <= b[1] - per < per          # a fixed tail, smaller than one candidate


def test_batch_workspace_holds_the_factors(gp):
    for n in (1, 127, 128, 129, 1000, 4000):
        per = {p: gp.call_bytes("nll_batch", n, 6, 2, p) - gp.call_bytes("nll_batch", n, 6, 1, p)
               for p in ("fp64", "mixed", "fp32")}
        # FP64: R's tiles in double; split: the double-float working matrix
        # and the copy of R the refinement residual reads
        assert per["fp64"] >= packed_bytes(n)
        assert per["mixed"] >= 2 * packed_bytes(n)
        # three slices of the factor take less than five
        assert per["fp32"] < per["mixed"]
        assert per["fp64"] < 2 * packed_bytes(n) + 64 * 1024


def test_auto_bounds_every_tier(gp):
    n, d, T = 2000, 6, 64
    tiers = [gp.call_bytes("nll_batch", n, d, T, p) for p in ("fp64", "mixed", "fp32")]
    auto = gp.call_bytes("nll_batch", n, d, T, "auto")
    assert auto >= max(tiers) + T * d * 8


def test_workspace_grows_with_n(gp):
    for call in ("nll_batch", "nll_grad"):
        sizes = [gp.call_bytes(call, n, 4, 3) for n in (100, 200, 400, 800, 1600)]
        assert sizes == sorted(sizes) and len(set(sizes)) == len(sizes)


def test_gradient_holds_three_triangles(gp):
    n, d = 1000, 6
    per = gp.call_bytes("nll_grad", n, d, 2) - gp.call_bytes("nll_grad", n, d, 1)
    assert per >= 3 * packed_bytes(n)   # the factor, L^-1 and R^-1


def test_fit_holds_the_factor_and_x(gp):
    for n, d in ((1, 1), (300, 3), (4064, 6)):
        m = gp.call_bytes("fit", n, d)
        f64 = gp.call_bytes("nll_batch", n, d, 1, "fp64")
        assert m >= packed_bytes(n) + n * d * 8
        assert m >= f64 + n * d * 8 - 256     # the FP64 instance plus the copy of x


def test_predict_scratch(gp):
    n, d = 1000, 6
    npad = 1024
    assert gp.call_bytes("predict", n, d, 0) == 0
    for N in (1, 100, 1000, 4000):
        # every point's solve column (a double-float pair per row) in one pass
        assert gp.call_bytes("predict", n, d, N) >= N * npad * 8
    # bounded in N: one wave of blocks, a second slot of r values and at most
    # 151 remainder blocks, whatever the number of points
    big = [gp.call_bytes("predict", n, d, N) for N in (100000, 200000, 10 ** 6, 2 ** 30)]
    assert max(big) <= 2 * gp.call_bytes("predict", n, d, 152 * 128) + 151 * npad * 128 * 8 * 4


def test_errors(gp):
    bad = [("nll_batch", 0, 6, 1, "mixed", gp.GP_EINVAL),
           ("nll_batch", 100, 0, 1, "mixed", gp.GP_EINVAL),
           ("nll_batch", 100, 65, 1, "mixed", gp.GP_EINVAL),
           ("nll_batch", 100, 6, 0, "mixed", gp.GP_EINVAL),
           ("nll_batch", 100, 6, 2 ** 30 + 1, "fp64", gp.GP_EINVAL),
           ("nll_grad", 100, 6, 2 ** 30 + 1, "fp64", gp.GP_EINVAL),
           ("nll_batch", 100, 6, 1, 9, gp.GP_EINVAL),
           ("nll_grad", 100, 17, 1, "fp64", gp.GP_ENOTSUP),
           ("predict", 100, 6, -1, "fp64", gp.GP_EINVAL),
           ("predict", 100, 6, 2 ** 30 + 1, "fp64", gp.GP_EINVAL)]
    for call, n, d, count, prec, code in bad:
        with pytest.raises(gp.GPError) as e:
            gp.call_bytes(call, n, d, count, prec)
        assert e.value.code == code, (call, n, d, count, prec)
    lib = gp.load()
    import ctypes
    out = ctypes.c_size_t()
    assert lib.gp_call_bytes(None, 7, 100, 6, 1, 1, ctypes.byref(out)) == gp.GP_EINVAL


def test_serving_admission_uses_the_library_sizes(gp):
    from paper_1203_1269_gb300 import serve
    for n, d in ((256, 2), (1000, 6), (8192, 12)):
        for prec in ("mixed", "fp64"):
            assert serve.eval_bytes(n, d, prec) == gp.call_bytes("nll_batch", n, d, serve.FIT_CANDIDATES, prec)
        assert serve.model_bytes(n, d) == gp.call_bytes("fit", n, d)
        assert serve.predict_bytes(n, d, 1000) == gp.call_bytes("predict", n, d, 1000)


def test_predict_workspace_of_the_tensor_core_path(gp):
    """The default predict path (predict_tc = 1): the slice tables of the
    factor (5 slices of the rows of L left of their diagonal blocks, 7 of each
    W_J = L_JJ^-1, three npad int arrays), an error flag, the r kernel's
    tables (2^(-j/1024) for j < 1024, 2^(m p) for |m| <= 60, F_j^p and 1/F_j
    for the 128 points F_j = 1 + j/128), per 128-point block
    of a chunk its r values (npad x 128 double-floats) and partial r'w
    (nt x 128), per CTA of the tensor-core pass the slices of V (5 x 4 nt
    chunks) and of C_J (7 x 4 chunks); a chunk is at most one wave of 152
    blocks.  Past one chunk the remainder blocks (blocks mod 152) get their
    own r values and CTA slices, and with two or more whole chunks the r
    values take a second slot."""
    al = lambda v: (v + 255) // 256 * 256
    chunk = 128 * 32 * 2
    rtab = al((1024 + 121 + 128) * 8 + 128 * 4)
    for n, d in ((1, 2), (300, 3), (4000, 6), (16384, 10)):
        nt = (n + 127) // 128
        npad = nt * 128
        tables = al(al(10 * nt * (nt - 1) * chunk) + al(nt * 28 * chunk) + 3 * al(npad * 4))
        per_block = npad * 128 * 8 + nt * 128 * 8
        per_cta = (5 * 4 * nt + 28) * chunk
        for N in (1, 128, 129, 5000, 152 * 128, 152 * 128 + 1, 2 * 152 * 128 + 300, 10 ** 6):
            blocks = (N + 127) // 128
            C = min(blocks, 152)
            rem = blocks % C if blocks > C else 0
            slots = 2 if rem > 0 and (blocks - rem) // C >= 2 else 1
            want = tables + 256 + rtab + slots * C * per_block + C * per_cta + rem * (per_block + per_cta)
            assert gp.call_bytes("predict", n, d, N) == want, (n, N)
