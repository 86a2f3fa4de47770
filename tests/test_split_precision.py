"""The arithmetic of the tensor-core gridding, emulated on the CPU (numpy):
per-sample power-of-two normalisation into [2^13, 2^14), FP16 hi / lo planes
of the samples and of the weights (with the factor 2^(a_ref - a) folded into
the weights), the three products hi.hi + hi.lo + lo.hi accumulated in FP32,
and the result times 2^-a_ref.  Checks that this is FP32-accurate: its error
against the FP64 sum is of the size of an FP32 sum's and far below that of
plain FP16 operands, with sample magnitudes spread over six decades within
one sum and whole scans scaled by 1e-30 or 1e30.  (The GPU tests compare the
kernels with the FP32 form; this pins the scheme itself.)"""
import numpy as np


def split16(x):
    hi = x.astype(np.float16)
    lo = (x - hi.astype(np.float32)).astype(np.float16)
    return hi, lo


def norm_exponent(bound):
    """a with bound * 2^a in [2^13, 2^14); an all-zero sample gets 127 (the
    largest exponent, so that it never sets the scan's reference a_ref)."""
    a = np.full(bound.shape, 127, np.int32)
    nz = bound > 0
    e = np.frexp(bound[nz].astype(np.float64))[1]   # bound = m 2^e, m in [0.5, 1)
    a[nz] = 14 - e
    return a


def split_gridding(s, w):
    """sum_l w[c, l] s[l, f] the tensor-core way.  s: [K, F] complex64,
    w: [C, K] float32.  Returns [C, F] complex64."""
    K = s.shape[0]
    sr = np.stack([s.real, s.imag], axis=-1).reshape(K, -1).astype(np.float32)   # [K, 2F]
    bound = np.sqrt(2.0) * np.abs(sr).max(axis=1)
    a = norm_exponent(bound)
    a_ref = a.min()
    sn = (sr * np.ldexp(np.float32(1), a)[:, None]).astype(np.float32)
    s_hi, s_lo = split16(sn)
    wn = (w * np.ldexp(np.float32(1), a_ref - a)[None, :]).astype(np.float32)
    w_hi, w_lo = split16(wn)
    f32 = lambda x: x.astype(np.float32)
    acc = np.zeros((w.shape[0], sr.shape[1]), np.float32)
    for k0 in range(0, K, 16):   # K steps of 16, three products each, FP32 accumulation
        ks = slice(k0, k0 + 16)
        acc += f32(w_hi[:, ks]) @ f32(s_hi[ks])
        acc += f32(w_lo[:, ks]) @ f32(s_hi[ks])
        acc += f32(w_hi[:, ks]) @ f32(s_lo[ks])
    acc = acc * np.ldexp(np.float32(1), -a_ref)
    out = acc.reshape(w.shape[0], -1, 2)
    return (out[..., 0] + 1j * out[..., 1]).astype(np.complex64)


def nmse(x, ref):
    return float(np.sum(np.abs(x - ref) ** 2) / np.sum(np.abs(ref) ** 2))


def _case(seed, K=300, C=64, F=64, spread=0.0):
    rng = np.random.default_rng(seed)
    s = (rng.standard_normal((K, F)) + 1j * rng.standard_normal((K, F))).astype(np.complex64)
    if spread:
        s *= np.power(10.0, rng.uniform(-spread, spread, K))[:, None].astype(np.float32)
    # Gaussian weights of a w = 6 kernel on an 8 x 8 tile: most are zero
    w = np.where(rng.random((C, K)) < 0.21, np.exp(-rng.uniform(0, 9, (C, K))), 0.0).astype(np.float32)
    return s, w


def test_split_products_are_fp32_accurate():
    for seed in range(4):
        s, w = _case(seed)
        ref = w.astype(np.float64) @ s.astype(np.complex128)
        got = split_gridding(s, w)
        fp32 = (w @ s).astype(np.complex64)                 # FP32 operands and sums
        fp16 = (w.astype(np.float16).astype(np.float32) @   # plain FP16 operands, FP32 sums
                (s.real.astype(np.float16).astype(np.float32) + 1j * s.imag.astype(np.float16).astype(np.float32)))
        e_split, e32, e16 = nmse(got, ref), nmse(fp32, ref), nmse(fp16, ref)
        assert e_split < 10 * max(e32, 1e-15), (e_split, e32)
        assert e_split < 1e-11, e_split
        assert e16 > 1e3 * e_split, (e16, e_split)   # the split is what buys the accuracy


def test_split_products_keep_accuracy_over_magnitudes():
    """Samples spanning 1e-3 .. 1e3 in one sum (each sample normalised by its
    own power of two) and whole scans scaled by 1e-30 or 1e30."""
    s, w = _case(7, spread=3.0)
    ref = w.astype(np.float64) @ s.astype(np.complex128)
    assert nmse(split_gridding(s, w), ref) < 1e-11
    s0, w0 = _case(8)
    base = split_gridding(s0, w0)
    for f in (1e-30, 1e30):
        scaled = split_gridding((s0 * np.float32(f)).astype(np.complex64), w0)
        assert nmse(scaled / f, base) < 1e-12, f


def test_zero_samples_and_zero_weights():
    s, w = _case(9, K=40)
    s[::3] = 0
    w[:, 5:9] = 0
    ref = w.astype(np.float64) @ s.astype(np.complex128)
    assert nmse(split_gridding(s, w), ref) < 1e-11
    assert np.all(split_gridding(np.zeros_like(s), w) == 0)
