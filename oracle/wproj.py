"""FP64 oracle of the W-projection hot path (test infrastructure; see package docstring).

Notation: N grid size, delta cell (rad), L = N delta field width, du = 1/L wavelengths
per cell, Nw w-planes, S_p full support of plane p (taps per axis, the paper's "full
support size", Sec. 2.2 and Sec. 3.1), os oversampling, M screen lattice size.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np
import scipy.special

C_LIGHT = 299792458.0


@dataclass(frozen=True)
class Params:
    """Imaging parameters (Sec. 3.1 lists image size, cell size, number of w-planes and
    full support; oversampling and the taper come from the W-projection method)."""
    n: int
    cell: float
    n_w: int
    w_max: float
    s_min: int
    s_max: int
    os: int
    m: int = 0          # screen lattice; 0 -> default_screen_m(s_max)

    @property
    def field(self) -> float:
        return self.n * self.cell

    @property
    def screen_m(self) -> int:
        return self.m if self.m > 0 else default_screen_m(self.s_max)


def plane_supports(n_w: int, s_min: int, s_max: int) -> np.ndarray:
    """Full support per plane, S_p = S_min + rint((S_max - S_min) p / (Nw - 1)).

    The paper uses one full support (9, Sec. 3.1) for all 23 planes; w-dependent support
    (larger kernels for larger |w|) is the reading used for the support ranges of the
    workloads. With S_min == S_max it reduces to the paper's single support.
    """
    if n_w == 1:
        return np.array([s_min], dtype=np.int64)
    p = np.arange(n_w)
    return (s_min + np.rint((s_max - s_min) * p / (n_w - 1))).astype(np.int64)


def plane_w(n_w: int, w_max: float) -> np.ndarray:
    """w of plane p (wavelengths): planes linear in |w|, w_p = p * (w_max / (Nw - 1))."""
    if n_w == 1:
        return np.zeros(1)
    return np.arange(n_w) * (w_max / (n_w - 1))


def default_screen_m(s_max: int) -> int:
    """Screen lattice size M (odd): 4 * S_max + 1, at least 65.

    An odd lattice is symmetric about l = 0, so the screen is exactly even in l and in m
    and never touches |x| = 1; the kernel is then exactly even and C_{-w} = conj(C_w).
    """
    return max(65, 4 * s_max + 1)


def taper_c(s_min: int) -> float:
    """PSWF bandwidth c = pi * S_min / 2 (its transform is confined to S_min cells)."""
    return math.pi * s_min / 2.0


_GL_NODES, _GL_WEIGHTS = np.polynomial.legendre.leggauss(256)


def taper(x, c: float) -> np.ndarray:
    """Anti-aliasing taper t(x) = psi_0(c, x) / psi_0(c, 0) on |x| <= 1 (x = l / (L/2)).

    psi_0 is the zeroth prolate spheroidal wave function (scipy.special.pro_ang1). That
    routine returns NaN at |x| = 1 exactly; there the value is taken from the defining
    integral equation int_{-1}^{1} exp(i c x y) psi(y) dy = lambda psi(x) at x = 1, with
    lambda fixed by the same equation at x = 0 (256-point Gauss-Legendre quadrature on
    interior nodes). psi_0 is even, so t(-1) = t(1).
    """
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    if np.any(ax > 1.0):
        raise ValueError("taper argument outside [-1, 1]")
    psi0 = scipy.special.pro_ang1(0, 0, c, 0.0)[0]
    out = np.empty_like(x)
    inner = ax < 1.0
    out[inner] = scipy.special.pro_ang1(0, 0, c, ax[inner])[0] / psi0
    if np.any(~inner):
        py = scipy.special.pro_ang1(0, 0, c, _GL_NODES)[0]
        lam = np.sum(_GL_WEIGHTS * py) / psi0
        edge = np.sum(_GL_WEIGHTS * np.cos(c * _GL_NODES) * py) / lam / psi0
        out[~inner] = edge
    return out


def screen(w: float, m: int, field: float, c: float) -> np.ndarray:
    """Image-plane screen of one w-plane on the M x M lattice, [q][k] (row = m, column = l).

        s(l_k, m_q) = t(x_k) t(x_q) exp(2 pi i w (n - 1)),  n = sqrt(1 - l^2 - m^2)
        l_k = j_k L / M,  x_k = 2 j_k / M,  j_k = k - (M - 1)/2  (M odd)

    The w-term phase screen times the taper (the W-projection kernel's image-plane form;
    the paper defers its definition to Cornwell et al. 2008, Sec. 1). n - 1 is formed as
    -r^2 / (1 + sqrt(1 - r^2)), which equals sqrt(1 - r^2) - 1 without cancellation.
    """
    if m % 2 == 0:
        raise ValueError("screen lattice size M must be odd")
    j = np.arange(m) - (m - 1) // 2
    x = 2.0 * j / m
    lk = j * field / m
    t = taper(x, c)
    r2 = lk[None, :] ** 2 + lk[:, None] ** 2
    if np.any(r2 >= 1.0):
        raise ValueError("field too wide: l^2 + m^2 >= 1 on the screen lattice")
    nm1 = -r2 / (1.0 + np.sqrt(1.0 - r2))
    return np.outer(t, t) * np.exp(2j * np.pi * w * nm1)


def wkernel_unnormalised(w: float, s: int, os_: int, m: int, field: float, c: float) -> np.ndarray:
    """Oversampled W-kernel of one plane before normalisation, [ey][ex] with E = S*os.

        K(dx, dy) = sum_{k,q} s(l_k, m_q) exp(-2 pi i (dx j_k + dy j_q) / (os M))

    for dx, dy in (-S os/2, S os/2] (1/os-cell offsets), stored at e = d + S os/2 - 1.
    Computed as the zero-padded os*M-point FFT of the centred screen (numpy.fft.fft2).
    """
    if (s * os_) % 2:
        raise ValueError("S * os must be even")
    big = os_ * m
    half = s * os_ // 2
    buf = np.zeros((big, big), np.complex128)
    idx = (np.arange(m) - (m - 1) // 2) % big
    buf[np.ix_(idx, idx)] = screen(w, m, field, c)
    f = np.fft.fft2(buf)
    d = np.arange(-half + 1, half + 1) % big
    return f[np.ix_(d, d)]


def wkernel_dft_bruteforce(w: float, s: int, os_: int, m: int, field: float, c: float) -> np.ndarray:
    """The same kernel by the direct double sum (pin for the FFT route; small M only)."""
    half = s * os_ // 2
    scr = screen(w, m, field, c)
    j = np.arange(m) - (m - 1) // 2
    d = np.arange(-half + 1, half + 1)
    ph = np.exp(-2j * np.pi * np.outer(d, j) / (os_ * m))      # [d][k]
    return ph @ scr @ ph.T                                      # [dy][dx]


def wkernels(prm: Params) -> tuple[list[np.ndarray], float]:
    """All planes' kernels, normalised, and the norm.

    Normalisation: divide every plane by nu = Re sum of the plane-0 taps at offsets that
    are whole cells (d = 0 mod os), i.e. the taps a w = 0 visibility lying exactly on a
    cell centre uses. Its kernel then sums to 1, so the grid sum of such a visibility is
    its value.
    """
    sup = plane_supports(prm.n_w, prm.s_min, prm.s_max)
    wp = plane_w(prm.n_w, prm.w_max)
    c = taper_c(prm.s_min)
    m = prm.screen_m
    raw = [wkernel_unnormalised(wp[p], int(sup[p]), prm.os, m, prm.field, c) for p in range(prm.n_w)]
    s0 = int(sup[0])
    half0 = s0 * prm.os // 2
    d = np.arange(-half0 + 1, half0 + 1)
    on_cell = np.nonzero(d % prm.os == 0)[0]
    nu = float(np.real(raw[0][np.ix_(on_cell, on_cell)].sum()))
    return [k / nu for k in raw], nu


def coords(uvw: np.ndarray, freqs: np.ndarray, prm: Params, hermitian_pairs: bool = False) -> dict:
    """uvw (m) -> per gridded visibility: plane, oversampled position, footprint, keep flag.

    For row r, channel c (s_c = f_c / c_light wavelengths per metre):
        kx_c = s_c * (os * (N * delta))        kw_c = s_c * ((Nw - 1) / w_max)
        U = rint(u_m * kx_c)   V = rint(v_m * kx_c)   (1/os-cell units; u/du*os)
        p = min(Nw - 1, rint(|w_m| * kw_c))    conj = (w_m < 0)
        X = U + (N/2) os,  i0 = floor((X - S_p os/2) / os) + 1,  ox = i0 os - X + S_p os/2 - 1
    (same for V, j0, oy). Footprint cells are i0 .. i0 + S_p - 1, i.e. the cells i with
    -S_p os/2 < i os - X <= S_p os/2. A visibility is kept if its footprint lies inside
    [0, N)^2 and its coordinates are finite with |U|, |V| < 2^30; others are dropped.
    rint is round-half-to-even, all in float64 (the GPU takes the same decisions in float64).
    With hermitian_pairs every sample is also gridded as its conjugate at -uvw
    (U -> -U, V -> -V, same plane, conj = (w_m > 0)), listed after all originals.
    Order: k = row * nchan + chan (+ nrow*nchan for the pairs).
    """
    uvw = np.asarray(uvw, dtype=np.float64)
    freqs = np.asarray(freqs, dtype=np.float64)
    n, os_ = prm.n, prm.os
    s = freqs / C_LIGHT
    kx = s * (os_ * (n * prm.cell))
    kw = s * ((prm.n_w - 1) / prm.w_max) if prm.n_w > 1 else np.zeros_like(s)
    with np.errstate(invalid="ignore", over="ignore"):
        ux = (uvw[:, 0:1] * kx[None, :]).ravel()
        vy = (uvw[:, 1:2] * kx[None, :]).ravel()
        wz = (np.abs(uvw[:, 2:3]) * kw[None, :]).ravel()
        wneg = np.broadcast_to(uvw[:, 2:3] < 0, (uvw.shape[0], len(freqs))).ravel()
        wpos = np.broadcast_to(uvw[:, 2:3] > 0, (uvw.shape[0], len(freqs))).ravel()
        finite = np.isfinite(ux) & np.isfinite(vy) & np.isfinite(wz)
        finite &= (np.abs(ux) < 2.0 ** 30) & (np.abs(vy) < 2.0 ** 30)
        u_i = np.where(finite, np.rint(ux), 0).astype(np.int64)
        v_i = np.where(finite, np.rint(vy), 0).astype(np.int64)
        pl = np.where(finite, np.minimum(prm.n_w - 1, np.rint(np.minimum(wz, 2.0 ** 30))), 0).astype(np.int64)
    if hermitian_pairs:
        u_i = np.concatenate([u_i, -u_i])
        v_i = np.concatenate([v_i, -v_i])
        pl = np.concatenate([pl, pl])
        conj = np.concatenate([wneg, wpos])
        finite = np.concatenate([finite, finite])
    else:
        conj = wneg.copy()
    sup = plane_supports(prm.n_w, prm.s_min, prm.s_max)[pl]
    half = sup * os_ // 2
    x = u_i + (n // 2) * os_
    y = v_i + (n // 2) * os_
    i0 = (x - half) // os_ + 1
    j0 = (y - half) // os_ + 1
    ox = i0 * os_ - x + half - 1
    oy = j0 * os_ - y + half - 1
    keep = finite & (i0 >= 0) & (i0 + sup <= n) & (j0 >= 0) & (j0 + sup <= n)
    return dict(U=u_i, V=v_i, plane=pl, conj=conj, support=sup, i0=i0, j0=j0, ox=ox, oy=oy,
                keep=keep, nvis=uvw.shape[0] * len(freqs), pairs=hermitian_pairs)


def gridded_values(vis: np.ndarray, weight: np.ndarray | None, crd: dict) -> np.ndarray:
    """c_k = W_k V_k (complex128); the Hermitian partner of a sample carries W_k conj(V_k)."""
    v = np.asarray(vis).astype(np.complex128).ravel()
    w = np.ones(v.shape) if weight is None else np.asarray(weight, dtype=np.float64).ravel()
    c = w * v
    if crd["pairs"]:
        c = np.concatenate([c, w * np.conj(v)])
    return c


def sum_weights(weight: np.ndarray | None, crd: dict) -> float:
    """Natural weighting: sum of the weights of every kept gridded visibility."""
    n = crd["nvis"]
    w = np.ones(n) if weight is None else np.asarray(weight, dtype=np.float64).ravel()
    if crd["pairs"]:
        w = np.concatenate([w, w])
    return float(np.sum(w[crd["keep"]]))


_LIB = None
_LIB_LOCK = threading.Lock()
_HERE = os.path.dirname(os.path.abspath(__file__))


def build_lib(force: bool = False) -> str:
    """Compile cgrid.c (plain C, OpenMP) into liboracle_cgrid.so next to it."""
    src = os.path.join(_HERE, "cgrid.c")
    out = os.path.join(_HERE, "liboracle_cgrid.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                        "-o", tmp, src], check=True)
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LIB_LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build_lib())
            p = ctypes.c_void_p
            lib.oracle_grid.argtypes = [ctypes.c_int64] + [p] * 10 + [ctypes.c_int32, ctypes.c_int32, p, ctypes.c_int32]
            lib.oracle_grid.restype = ctypes.c_int
            lib.oracle_degrid.argtypes = [ctypes.c_int64] + [p] * 9 + [ctypes.c_int32, ctypes.c_int32, p, p, ctypes.c_int32]
            lib.oracle_degrid.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def _packed_tables(tables: list[np.ndarray]):
    offs = np.zeros(len(tables), np.int64)
    acc = 0
    for p, t in enumerate(tables):
        offs[p] = acc
        acc += t.size
    flat = np.concatenate([np.ascontiguousarray(t, np.complex128).ravel() for t in tables])
    return offs, flat


def _kept_arrays(crd: dict):
    kp = crd["keep"]
    a = [np.ascontiguousarray(crd[k][kp], np.int32) for k in ("i0", "j0", "ox", "oy", "plane")]
    cj = np.ascontiguousarray(crd["conj"][kp], np.uint8)
    return kp, a, cj


def grid(crd: dict, c: np.ndarray, tables: list[np.ndarray], prm: Params, threads: int = 1) -> np.ndarray:
    """Gridding: G[j0+b, i0+a] += c_k K_k[b os + oy, a os + ox] over kept visibilities, FP64."""
    kp, (i0, j0, ox, oy, pl), cj = _kept_arrays(crd)
    ck = np.ascontiguousarray(np.asarray(c, np.complex128)[kp])
    offs, flat = _packed_tables(tables)
    sup = plane_supports(prm.n_w, prm.s_min, prm.s_max).astype(np.int32)
    g = np.zeros((prm.n, prm.n), np.complex128)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    rc = _lib().oracle_grid(len(ck), ptr(i0), ptr(j0), ptr(ox), ptr(oy), ptr(pl), ptr(cj), ptr(ck),
                            ptr(sup), ptr(offs), ptr(flat), prm.os, prm.n, ptr(g), threads)
    if rc:
        raise MemoryError("oracle_grid: private grid allocation failed")
    return g


def degrid(crd: dict, g: np.ndarray, tables: list[np.ndarray], prm: Params, threads: int = 1) -> np.ndarray:
    """Degridding (adjoint of `grid` with unit weights); dropped visibilities get 0.

    Returns complex128 of length nvis (x2 with Hermitian pairs) in coords() order.
    """
    kp, (i0, j0, ox, oy, pl), cj = _kept_arrays(crd)
    offs, flat = _packed_tables(tables)
    sup = plane_supports(prm.n_w, prm.s_min, prm.s_max).astype(np.int32)
    gg = np.ascontiguousarray(np.asarray(g, np.complex128))
    out = np.zeros(int(kp.sum()), np.complex128)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _lib().oracle_degrid(len(out), ptr(i0), ptr(j0), ptr(ox), ptr(oy), ptr(pl), ptr(cj), ptr(sup),
                         ptr(offs), ptr(flat), prm.os, prm.n, ptr(gg), ptr(out), threads)
    full = np.zeros(kp.shape, np.complex128)
    full[kp] = out
    return full


def fft_to_image(g: np.ndarray, sum_w: float, prm: Params, taper_correct: bool = True) -> np.ndarray:
    """Dirty image from the grid (the IFFT step, Fig. 1 and Fig. 2 captions), then the
    taper correction:
        I[j, i] = Re sum_{h,g} G[h, g] exp(+2 pi i ((g - N/2)(i - N/2) + (h - N/2)(j - N/2)) / N)
        I[j, i] /= sum_w * t(x_i) t(x_j),   x_i = 2 (i - N/2) / N
    (without the taper factor when taper_correct is False). Computed as
    Re(fftshift(ifft2(ifftshift(G))) * N^2)."""
    n = g.shape[0]
    f = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(g))) * (n * n)
    img = f.real / sum_w
    if taper_correct:
        x = 2.0 * (np.arange(n) - n // 2) / n
        t = taper(x, taper_c(prm.s_min))
        img = img / np.outer(t, t)
    return img


def image_to_grid_adjoint(img: np.ndarray, sum_w: float, prm: Params, taper_correct: bool = True) -> np.ndarray:
    """Adjoint of fft_to_image as a real-linear map from the complex grid to the real image:
    <fft_to_image(G), X> = Re <G, image_to_grid_adjoint(X)>."""
    n = img.shape[0]
    x = np.asarray(img, np.float64) / sum_w
    if taper_correct:
        xs = 2.0 * (np.arange(n) - n // 2) / n
        t = taper(xs, taper_c(prm.s_min))
        x = x / np.outer(t, t)
    # I = Re(A G) with A the centred unnormalised inverse DFT; adjoint of G -> Re(A G) is X -> A^H X
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(x)))


def dirty_image_dft(uvw: np.ndarray, freqs: np.ndarray, c: np.ndarray, n: int, cell: float,
                    w_exact: bool = True, pixels: np.ndarray | None = None) -> np.ndarray:
    """Direct-DFT dirty image (no gridding, no kernels), the quantity W-projection approximates:
        I_D[j, i] = Re sum_k c_k exp(+2 pi i (u_k l_i + v_k m_j + w_k (n_ij - 1)))
    with l_i = (i - N/2) delta, m_j = (j - N/2) delta, u, v, w in wavelengths and
    c_k = W_k V_k (not divided by the weight sum). `pixels` optionally restricts the
    evaluation to an [npix, 2] array of (j, i)."""
    uvw = np.asarray(uvw, np.float64)
    s = np.asarray(freqs, np.float64) / C_LIGHT
    u = (uvw[:, 0:1] * s).ravel()
    v = (uvw[:, 1:2] * s).ravel()
    w = (uvw[:, 2:3] * s).ravel()
    c = np.asarray(c, np.complex128).ravel()
    if pixels is None:
        jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        pix = np.stack([jj.ravel(), ii.ravel()], axis=1)
    else:
        pix = np.asarray(pixels)
    lm = (pix - n // 2) * cell
    lv, mv = lm[:, 1], lm[:, 0]
    r2 = lv * lv + mv * mv
    nm1 = -r2 / (1.0 + np.sqrt(1.0 - r2)) if w_exact else np.zeros_like(r2)
    out = np.empty(len(pix))
    for s0 in range(0, len(pix), 256):
        sl = slice(s0, s0 + 256)
        ph = np.outer(lv[sl], u) + np.outer(mv[sl], v) + np.outer(nm1[sl], w)
        out[sl] = np.real(np.exp(2j * np.pi * ph) @ c)
    return out.reshape(n, n) if pixels is None else out
