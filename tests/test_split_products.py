"""The operand splits of the tensor-core precisions, checked on the host in
numpy: ADG_PREC_MIXED_TF32 keeps the top 11 significant bits of an FP32
operand (its TF32 part) and the exact FP32 remainder; ADG_PREC_MIXED_BF16X3
splits an FP32 operand into three BF16 numbers, each the top 8 significant
bits of what remains.  Both splits are exact (the parts sum to the operand
with no rounding).  The products the kernels keep leave the errors their
comments state: for TF32 (whose MMA reads the remainders as TF32 too) about
2^-19 of the product at worst and 2^-22 typically, for BF16x3 about 2^-21 at
worst and 2^-25 typically, against 2^-24 for one FP32 rounding."""
import numpy as np


def _f32(bits):
    return np.asarray(bits, dtype=np.uint32).view(np.float32)


def _bits(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def tf32_split(a):
    hi = _f32(_bits(a) & np.uint32(0xFFFFE000))
    lo = (a - hi).astype(np.float32)
    return hi, lo


def bf16_split3(a):
    hi = _f32(_bits(a) & np.uint32(0xFFFF0000))
    r1 = (a - hi).astype(np.float32)
    mid = _f32(_bits(r1) & np.uint32(0xFFFF0000))
    r2 = (r1 - mid).astype(np.float32)
    lo = _f32(_bits(r2) & np.uint32(0xFFFF0000))
    return hi, mid, lo, r2


def _operands(seed, k=200000):
    rng = np.random.default_rng(seed)
    mag = np.exp(rng.uniform(np.log(1e-6), np.log(1e6), k))
    return (rng.choice([-1.0, 1.0], k) * mag).astype(np.float32)


def test_bf16_three_way_split_is_exact():
    a = _operands(1)
    hi, mid, lo, r2 = bf16_split3(a)
    # each part is a BF16 number (low 16 bits of its FP32 pattern zero)
    for p in (hi, mid, lo):
        assert not np.any(_bits(p) & np.uint32(0xFFFF))
    # the last remainder already fits in BF16, so nothing is dropped
    assert np.array_equal(lo, r2)
    # exact: summed in FP64 the parts give the operand bit for bit
    s = hi.astype(np.float64) + mid.astype(np.float64) + lo.astype(np.float64)
    assert np.array_equal(s, a.astype(np.float64))


def test_tf32_split_is_exact():
    a = _operands(2)
    hi, lo = tf32_split(a)
    assert not np.any(_bits(hi) & np.uint32(0x1FFF))
    assert np.array_equal(hi.astype(np.float64) + lo.astype(np.float64), a.astype(np.float64))


def _tf32_read(x):
    """What a TF32 MMA reads from an FP32 register: its top 19 bits."""
    return _f32(_bits(x) & np.uint32(0xFFFFE000))


def test_kept_products_error_order():
    """Products of two split operands, the kept terms summed in FP64."""
    a, d = _operands(3), _operands(4)
    exact = a.astype(np.float64) * d.astype(np.float64)
    f = lambda x: x.astype(np.float64)
    ah, am, al, _ = bf16_split3(a)
    dh, dm, dl, _ = bf16_split3(d)
    bf = f(ah) * f(dh) + f(am) * f(dh) + f(ah) * f(dm) + f(al) * f(dh) + f(am) * f(dm) + f(ah) * f(dl)
    rel_bf = np.abs(bf - exact) / np.abs(exact)
    assert rel_bf.max() <= 2.0 ** -20 and np.median(rel_bf) <= 2.0 ** -24, (rel_bf.max(), np.median(rel_bf))
    th, tl = tf32_split(a)
    eh, el = tf32_split(d)
    tf = f(_tf32_read(tl)) * f(eh) + f(th) * f(_tf32_read(el)) + f(th) * f(eh)
    rel_tf = np.abs(tf - exact) / np.abs(exact)
    assert rel_tf.max() <= 2.0 ** -18 and np.median(rel_tf) <= 2.0 ** -21, (rel_tf.max(), np.median(rel_tf))
    # each kept term matters: without a_hi d_lo (order 2^-14) the BF16x3
    # error grows to about 2^-15, without a_lo d_hi the TF32 one to 2^-11
    assert (np.abs(bf - f(ah) * f(dl) - exact) / np.abs(exact)).max() > 2.0 ** -17
    assert (np.abs(tf - f(_tf32_read(tl)) * f(eh) - exact) / np.abs(exact)).max() > 2.0 ** -13
