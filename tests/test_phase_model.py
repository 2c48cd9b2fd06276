"""Host model of the tensor-core synthesis phase (no GPU).

The synthesis kernels form frac(<r, q>) (r a unit pixel vector, q = p / wl in
wavelengths) from 32-bit integer station words and FP32 corrections:
per component r = R 2^-29 + rl and q = QH / 8 + ql with R, QH 32-bit integers,
so that r q = R QH 2^-32 + r ql + rl q - rl ql, the first term taken as the
wrapped 32-bit product. This file re-enacts that arithmetic in numpy (int32
wrap-around, FP32 rounding of every operation the kernel does in FP32) and
checks it against the phase computed in exact rational arithmetic from the same
FP64 inputs: the error stays near the 2^-25 cycles of the FP32 rounding of the
fraction, over baselines up to 65 km and far beyond, and the kernel's radian
argument stays within the range its sincos is used on.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

TWO_PI = 6.283185307179586


def _words(q):
    """k_tc_pack: QH = round(8 q) (32-bit), 2 pi ql and 2 pi q in FP32."""
    q8 = np.rint(8.0 * q)
    QH = q8.astype(np.int64)
    ql = np.float32(TWO_PI * (q - 0.125 * q8))
    qf = np.float32(TWO_PI * q)
    return QH, ql, qf


def _pix(r):
    """phase_pix: R = round(r 2^29), r and rl = r - R 2^-29 in FP32."""
    R = np.rint(r * 536870912.0).astype(np.int64)
    return R, np.float32(r), np.float32(r - R * 1.862645149230957e-09)


def _fma32(a, b, c):
    """An FP32 FMA: the product of two floats is exact in FP64, one rounding to FP32."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _kernel_phase(r, q):
    """The kernel's radian argument for one pixel (3,) and stations (n, 3)."""
    R, rf, rl = _pix(r)
    QH, ql, qf = _words(q)
    acc = np.zeros(q.shape[0], dtype=np.int64)
    for c in range(3):
        acc = (acc + R[c] * QH[:, c]) % (1 << 32)  # 32-bit IMADs: wrap-around
    acc = np.where(acc >= (1 << 31), acc - (1 << 32), acc)
    f = np.float32(np.float64(rf[0]) * np.float64(ql[:, 0]))  # FMUL
    f = _fma32(rf[1], ql[:, 1], f)
    f = _fma32(rf[2], ql[:, 2], f)
    for c in range(3):
        f = _fma32(rl[c], qf[:, c], f)
    k = np.float32(1.4629180792671596e-09)  # 2 pi 2^-32
    return _fma32(np.float32(acc), k, f)  # I2F, then the combining FMA


def _exact_cycles(r, q):
    """frac(<r, q>) in [-1/2, 1/2), exactly, from the FP64 inputs."""
    out = []
    for qi in q:
        s = sum(Fraction(float(r[c])) * Fraction(float(qi[c])) for c in range(3))
        fr = s - round(s)
        out.append(float(fr))
    return np.array(out)


def _wrap(x):
    return (x + 0.5) % 1.0 - 0.5


def _case(seed, q_scale, n=64):
    rng = np.random.default_rng(seed)
    r = rng.normal(size=3)
    r /= np.linalg.norm(r)
    q = rng.normal(size=(n, 3)) * q_scale
    return r, q


def test_phase_error_at_ska_baselines():
    # stations up to ~65 km at wl = 2 m: |q| up to ~3.3e4 wavelengths
    for seed in range(6):
        r, q = _case(seed, 3.3e4 / 3)
        got = _kernel_phase(r, q) / TWO_PI
        err = np.abs(_wrap(got - _exact_cycles(r, q)))
        assert err.max() < 2.0 ** -23, err.max()
        assert np.abs(_kernel_phase(r, q)).max() < 4.4  # the sincos argument range of the header comment


def test_phase_error_far_out():
    # stations up to 2^27 wavelengths from the origin (inside the 2^28 limit)
    for seed in range(4):
        r, q = _case(100 + seed, 2.0 ** 27 / 3)
        q = np.clip(q, -2.0 ** 27, 2.0 ** 27)
        got = _kernel_phase(r, q) / TWO_PI
        err = np.abs(_wrap(got - _exact_cycles(r, q)))
        assert err.max() < 2.0 ** -22, err.max()


def test_range_limit_of_the_integer_words():
    # 8 q must fit a signed 32-bit word: |q| < 2^28 wavelengths
    QH, _, _ = _words(np.array([[2.0 ** 28 - 1.0, 0.0, -(2.0 ** 28 - 1.0)]]))
    assert np.abs(QH).max() < 2 ** 31
