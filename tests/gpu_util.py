"""Shared helpers for the GPU parity tests (CUDA path vs the CPU oracle)."""
import math

import numpy as np

U32 = 2.0 ** -24          # unit roundoff of FP32


def bz_module():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2103_14890_gb300 import build, binding
    build.build()
    binding.load()
    return binding


def to_dev(a, precision):
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def as_input(a, precision):
    """The exact values the device sees, in FP64 (the oracle gets the same)."""
    return a if precision == "fp64" else a.astype(np.float32).astype(np.float64)


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class AbsModeSum:
    """Rounding-error scale of the collision operator (Sec. 3.3, eq. CF1).

    For every cell, A_k = sum over l + m = k in K_h of |beta(l,m)| |f-hat_l|
    |f-hat_m|: the mode sum with every term replaced by its magnitude.  Each
    rounding on the path (spectrum, weight, product, accumulation) perturbs a
    term by a multiple of u times its magnitude, so the error of Q-hat_k is a
    multiple of u A_k however strongly gain and loss cancel in Q-hat_k itself.
    The weights and spectra are the oracle's (FP64 kernel modes and naive
    DFT), never the library's."""

    def __init__(self, k):
        self.k = k
        M, h, d = k.M, k.h, k.dim
        idx = np.indices((M,) * d).reshape(d, -1).T - h          # mode vectors of the flat index
        nm = idx.shape[0]
        li, mi, ki = [], [], []
        for l in range(nm):
            kv = idx[l] + idx
            ok = np.nonzero((np.abs(kv) <= h).all(axis=1))[0]
            li.append(np.full(len(ok), l))
            mi.append(ok)
            ki.append(np.ravel_multi_index(tuple((kv[ok] + h).T), (M,) * d))
        self.li, self.mi, self.ki = np.concatenate(li), np.concatenate(mi), np.concatenate(ki)
        self.wabs = np.abs(k.beta_pairs(self.li, self.mi))
        self.nm = nm

    def __call__(self, f):
        """(n_cells, N^d) -> A of shape (n_cells, (2h+1)^d) (full spectrum)."""
        f = np.atleast_2d(f)
        out = np.empty((f.shape[0], self.nm))
        for c in range(f.shape[0]):
            a = np.abs(self.k.dft_forward(f[c])).ravel()
            out[c] = np.bincount(self.ki, self.wabs * a[self.li] * a[self.mi], minlength=self.nm)
        return out


def fp32_cell_bounds(k, A, Qr):
    """Per-cell bounds on the FP32 operator's error, from the rounding count.

    c_M = 2 log2(N^d) + 4 roundings of relative size u per term of the mode
    sum: log2(N^d) radix stages of the forward FFT on each of the two
    spectrum values, the weight, the scaled value w f-hat_l, the product's
    accumulation and the fold into the (hi, lo) pair.  The inverse FFT adds
    c_F = 2 log2(N^d) u of the result.  With Parseval (sum_j Q_j^2 =
    s^(2(d+gamma)) N^d sum_k |Q-hat_k|^2):
      L2 per cell:   |dQ|_2   <= u (c_M s^(d+gamma) sqrt(N^d) |A|_2 + c_F |Q|_2)
      any element:   |dQ_j|   <= u (c_M s^(d+gamma) |A|_1        + c_F |Q|_2)
    (the element bound is the triangle inequality over the inverse DFT).
    Returns (bound_l2, bound_inf), one entry per cell."""
    nv = k.N ** k.dim
    p = math.log2(nv)
    cM, cF = 2 * p + 4, 2 * p
    sdg = k.s ** (k.dim + k.gamma)
    qn = np.linalg.norm(Qr, axis=1)
    b2 = U32 * (cM * sdg * math.sqrt(nv) * np.linalg.norm(A, axis=1) + cF * qn)
    binf = U32 * (cM * sdg * np.abs(A).sum(axis=1) + cF * qn)
    return b2, binf


def check_fp32_cells(k, f_in, Q, Qr, A=None, what=""):
    """Assert the per-cell L2 and element-wise FP32 bounds; returns the largest
    ratios (error / bound) and the largest per-cell relative L2 error."""
    if A is None:
        A = AbsModeSum(k)(f_in)
    b2, binf = fp32_cell_bounds(k, A, Qr)
    d = Q - Qr
    e2 = np.linalg.norm(d, axis=1)
    einf = np.abs(d).max(axis=1)
    r2, rinf = e2 / b2, einf / binf
    rel = e2 / np.maximum(np.linalg.norm(Qr, axis=1), 1e-300)
    print("%s per-cell: worst L2/bound %.3f, worst max/bound %.3f, worst cell rel-L2 %.2e"
          % (what, r2.max(), rinf.max(), rel.max()))
    assert (r2 <= 1.0).all(), (what, int(np.argmax(r2)), float(r2.max()))
    assert (rinf <= 1.0).all(), (what, int(np.argmax(rinf)), float(rinf.max()))
    return float(r2.max()), float(rinf.max()), float(rel.max())
