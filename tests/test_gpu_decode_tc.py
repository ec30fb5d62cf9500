"""GPU parity of crom_decode_tc, Step 1 of the latent step on the tcgen05 tensor
cores (paper §4.1, Algorithm 4; Algorithm 2 for the spatial derivatives), against
the FP64 oracle's MLPDecoder, through the C ABI.

The kernel multiplies f16 copies of the hidden matrices and of W_1q (the Jacobian
projection), and f16 activations (hi/lo pairs at F16X2, single values at F16).  Two
comparisons per channel:
  * against the oracle evaluating the same f16-rounded matrices (the activation
    arithmetic alone): F16X2 carries ~2^-22 relative per layer input, F16 2^-12;
    the Laplacian loses about two digits to cancellation in the output layer;
  * against the oracle of the FP32 weights (what a user compares with): the
    weights' f16 rounding (2^-12) moves values by ~5e-4 and the Laplacian by up to
    ~1e-1 on these random decoders.
"""
import numpy as np
import pytest

from oracle import crom_oracle as O
from workloads import gen

from helpers import dev, make_ctx, rel_l2

pytestmark = pytest.mark.gpu

# tolerances (relative L2 per channel): against the f16-rounded matrices, per precision
# (dq: the reference rounds W_1q in the forward pass too, where the kernel keeps it in
# FP32; that difference alone is 2^-12-relative, about 1e-4 in J)
TOL_ROUNDED = {"CROM_PREC_F16X2": {"val": 1e-5, "dx": 1e-4, "lap": 1e-3, "dq": 5e-4},
               "CROM_PREC_F16": {"val": 3e-3, "dx": 1e-2, "lap": 1e-1, "dq": 1e-2}}
# against the FP32 weights: the weight rounding dominates at either precision
TOL_FP32 = {"val": 3e-3, "dx": 2e-2, "lap": 0.25, "dq": 2e-2}


@pytest.fixture(scope="module")
def c():
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    return crom


def f16_rounded(params, m, with_w1q):
    """The matrices the tensor-core path multiplies in f16: the hidden matrices
    (and W_1q for the Jacobian projection), rounded once; biases, W_1x and w_out stay."""
    out = []
    for l, (W, b) in enumerate(params):
        W = np.array(W, np.float64)
        if 0 < l < len(params) - 1:
            W = W.astype(np.float16).astype(np.float64)
        elif l == 0 and with_w1q:
            W[:, m:] = W[:, m:].astype(np.float16).astype(np.float64)
        out.append((W, np.array(b, np.float64)))
    return out


def run_decode(c, ctx, q, sizes, X, want, prec):
    import torch
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    rows = 0
    for bit, n in ((c.CROM_WANT_VAL, 1), (c.CROM_WANT_DX, X.shape[1]), (c.CROM_WANT_LAP, 1),
                   (c.CROM_WANT_DQ, q.shape[1])):
        rows += n if want & bit else 0
    out = torch.full((rows, X.shape[0]), np.nan, dtype=torch.float32, device="cuda")
    c.crom_decode_tc(ctx, dev(q, torch.float64), dev(off, torch.int32), dev(X, torch.float32), want, out,
                     precision=prec)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), off


def split_rows(out, m, r, want, c):
    res, k = {}, 0
    if want & c.CROM_WANT_VAL:
        res["val"] = out[k]; k += 1
    if want & c.CROM_WANT_DX:
        res["dx"] = out[k:k + m].T; k += m
    if want & c.CROM_WANT_LAP:
        res["lap"] = out[k]; k += 1
    if want & c.CROM_WANT_DQ:
        res["dq"] = out[k:k + r].T; k += r
    return res


def oracle_channels(params, m, X, Qp):
    ev = O.MLPDecoder(params, m)(X, Qp)
    return {"val": ev.g, "dx": ev.gx, "lap": ev.lap, "dq": ev.gq}


@pytest.mark.parametrize("prec_name", ["CROM_PREC_F16X2", "CROM_PREC_F16"])
@pytest.mark.parametrize("m,r,hidden", [(2, 8, 5), (1, 4, 3), (2, 15, 2)])
def test_decode_tc_matches_oracle(c, prec_name, m, r, hidden):
    """Ragged instances (an empty one, one point, sizes around the 256-point work
    chunks and the 16 / 32-sample tiles) on general FP32 weights; all channels."""
    spec = gen.DecoderSpec(m, r, 128, hidden)
    params = gen.xavier_decoder(spec, seed=31 + r + hidden, bias_std=0.1)
    ctx = make_ctx(spec, params)
    rng = np.random.default_rng(7 + m)
    sizes = [0, 1, 17, 255, 256, 257, 600, 33]
    X = rng.uniform(0.05, 0.95, size=(sum(sizes), m)).astype(np.float32)
    q = rng.standard_normal((len(sizes), r))
    want = c.CROM_WANT_VAL | c.CROM_WANT_DX | c.CROM_WANT_LAP | c.CROM_WANT_DQ
    out, off = run_decode(c, ctx, q, sizes, X, want, getattr(c, prec_name))
    assert np.all(np.isfinite(out))
    got = split_rows(out, m, r, want, c)
    Qp = np.repeat(q, sizes, axis=0)
    ref16 = oracle_channels(f16_rounded(params, m, False), m, X, Qp)
    ref16q = oracle_channels(f16_rounded(params, m, True), m, X, Qp)
    ref32 = oracle_channels(params, m, X, Qp)
    for ch in ("val", "dx", "lap", "dq"):
        e16 = rel_l2(got[ch], (ref16q if ch == "dq" else ref16)[ch])
        e32 = rel_l2(got[ch], ref32[ch])
        print(f"{prec_name} m={m} r={r} L={hidden} {ch}: vs f16 matrices {e16:.2e}, vs FP32 weights {e32:.2e}")
        assert e16 < TOL_ROUNDED[prec_name][ch], (ch, e16)
        assert e32 < TOL_FP32[ch], (ch, e32)
    ctx.close()


def test_decode_tc_channel_subsets_and_layout(c):
    """Rows appear in crom_decode's order for any subset; the reverse pass is skipped
    without DQ and the values do not change; DXX is refused."""
    import torch
    spec = gen.DecoderSpec(2, 6, 128, 4)
    params = gen.xavier_decoder(spec, seed=3, bias_std=0.1)
    ctx = make_ctx(spec, params)
    rng = np.random.default_rng(2)
    sizes = [40, 300]
    X = rng.uniform(0, 1, size=(sum(sizes), 2)).astype(np.float32)
    q = rng.standard_normal((2, 6))
    full_want = c.CROM_WANT_VAL | c.CROM_WANT_DX | c.CROM_WANT_LAP | c.CROM_WANT_DQ
    full, _ = run_decode(c, ctx, q, sizes, X, full_want, c.CROM_PREC_F16X2)
    full = split_rows(full, 2, 6, full_want, c)
    for want in (c.CROM_WANT_VAL, c.CROM_WANT_DQ, c.CROM_WANT_DX | c.CROM_WANT_LAP, c.CROM_WANT_VAL | c.CROM_WANT_DQ):
        out, _ = run_decode(c, ctx, q, sizes, X, want, c.CROM_PREC_F16X2)
        part = split_rows(out, 2, 6, want, c)
        for ch, v in part.items():
            assert np.array_equal(v, full[ch]), (want, ch)
    out = torch.zeros((3, X.shape[0]), dtype=torch.float32, device="cuda")
    with pytest.raises(c.CromError) as e:
        c.crom_decode_tc(ctx, dev(q, torch.float64), dev(np.array([0, 40, 340], np.int32), torch.int32),
                         dev(X, torch.float32), c.CROM_WANT_DXX, out)
    assert e.value.code == c.CROM_ERR_UNSUPPORTED
    assert c.crom_device_flags(ctx) == 0
    ctx.close()


def test_decode_tc_full_size_sampled(c):
    """All 273,723 integration samples of the 1024-instance workload in one launch;
    2000 sampled points recomputed by the oracle; the values agree with the FP32
    crom_decode."""
    import torch
    w = gen.heat2d_batched(n_inst=1024)
    ctx = make_ctx(w.spec, w.params)
    want = c.CROM_WANT_VAL | c.CROM_WANT_DX | c.CROM_WANT_LAP | c.CROM_WANT_DQ
    out, _ = run_decode(c, ctx, w.q0, w.sizes, w.samples, want, c.CROM_PREC_F16X2)
    assert np.all(np.isfinite(out))
    got = split_rows(out, 2, w.spec.r, want, c)
    idx = np.sort(np.random.default_rng(4).choice(w.samples.shape[0], size=2000, replace=False))
    Qp = np.repeat(w.q0, w.sizes, axis=0)[idx]
    ref16 = oracle_channels(f16_rounded(w.params, 2, False), 2, w.samples[idx], Qp)
    ref16q = oracle_channels(f16_rounded(w.params, 2, True), 2, w.samples[idx], Qp)
    for ch in ("val", "dx", "lap", "dq"):
        e16 = rel_l2(got[ch][idx], (ref16q if ch == "dq" else ref16)[ch])
        print(f"full size {ch}: vs f16 matrices {e16:.2e}")
        assert e16 < TOL_ROUNDED["CROM_PREC_F16X2"][ch], (ch, e16)
    off = dev(w.s_off, torch.int32)
    out32 = torch.empty((1, w.samples.shape[0]), dtype=torch.float32, device="cuda")
    c.crom_decode(ctx, dev(w.q0, torch.float64), off, dev(w.samples, torch.float32), c.CROM_WANT_VAL, out32)
    torch.cuda.synchronize()
    assert rel_l2(got["val"], out32.cpu().numpy()[0].astype(np.float64)) < TOL_FP32["val"]
    assert c.crom_device_flags(ctx) == 0
    ctx.close()
