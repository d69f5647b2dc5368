"""Frequency-domain model of the directional filter bank (test helper).

An independent route to the same transform the oracle computes by in-place
lifting: every lifting stage acting on a channel whose samples are
o + b1*p1 + b2*p2 is a pair of 2-D filters in the ORIGINAL frequency plane,

    W(w)  = sum_{a,b} betat[a] betat[b] exp(i w . (delta1 b1 + delta2 b2))
    F_odd  = (1 - W) / 2,      F_even = 1 + W * F_odd,

(delta = ((a+b)/2, (a-b)/2)).  A leaf subband is the product of the
filters along its tree path, applied by FFT to the whole plane, sampled on
the leaf's coset.  No lifting, no in-place update, no parity map: a
mistake in the oracle's offsets, parities, pass order or leaf extraction
shows up as a mismatch against this model.

The model also yields the wedge geometry of every leaf, used to check that
each subband's energy sits in its own wedge of the frequency plane (§2.1:
"2^l subbands with wedge-shaped frequency partitioning").
"""
import numpy as np

BETA_T = {-3: -1.0 / 16, -1: -9.0 / 16, 1: 9.0 / 16, 3: 1.0 / 16}


def lagrange_fan_taps(n):
    """Fan taps of the n-tap Lagrange half-band prototype, from the interpolation
    formula rather than a table: beta[a] is the weight of the sample at odd a in
    the polynomial interpolation of degree n - 1 evaluated at 0, i.e.
    prod_{b != a} b / (b - a), then modulated to the fan by (-1)^((a - 1) / 2)."""
    pts = list(range(-(n - 1), n, 2))
    taps = {}
    for a in pts:
        w = 1.0
        for b in pts:
            if b != a:
                w *= b / (b - a)
        taps[a] = (-1.0) ** (((a - 1) // 2) % 2) * w
    return taps


def basis(s, T, i):
    if s == 1:
        return (1, 0), (0, 1)
    if s == 2:
        return ((1, 1), (1, -1)) if T == "c" else ((1, 1), (-1, 1))
    q = 2 ** (s - 2)
    return ((q, -2 * i), (q, -2 * i - 2)) if T == "c" else ((-2 * i, q), (-2 * i - 2, q))


def leaves(H, W, k, taps=None):
    """Leaf list in tree order: dict(o, T, i, F) with F the equivalent filter on the DFT grid."""
    taps = BETA_T if taps is None else taps
    wr = 2 * np.pi * np.fft.fftfreq(H)[:, None]
    wc = 2 * np.pi * np.fft.fftfreq(W)[None, :]
    chans = [dict(o=(0, 0), T=None, i=None, F=np.ones((H, W), complex))]
    for s in range(1, k + 1):
        new = []
        for ch in chans:
            (b1r, b1c), (b2r, b2c) = basis(s, ch["T"], ch["i"])
            Wf = np.zeros((H, W), complex)
            for a, ba in taps.items():
                for b, bb in taps.items():
                    d1, d2 = (a + b) // 2, (a - b) // 2
                    Wf += ba * bb * np.exp(1j * (wr * (d1 * b1r + d2 * b2r) + wc * (d1 * b1c + d2 * b2c)))
            Fo = 0.5 * (1 - Wf)
            Fe = 1 + Wf * Fo
            o = ch["o"]
            o1 = (o[0] + b1r, o[1] + b1c)
            if s == 1:
                kids = (("c", None), ("r", None))
            elif s == 2:
                kids = ((ch["T"], -1), (ch["T"], 0))
            else:
                kids = ((ch["T"], 2 * ch["i"]), (ch["T"], 2 * ch["i"] + 1))
            new.append(dict(o=o, T=kids[0][0], i=kids[0][1], F=ch["F"] * Fe))
            new.append(dict(o=o1, T=kids[1][0], i=kids[1][1], F=ch["F"] * Fo))
        chans = new
    return chans, wr, wc


def analysis(x, k, taps=None):
    """Concatenated subbands of plane x (tree order), computed by FFT filtering."""
    H, W = x.shape
    X = np.fft.fft2(x)
    out = []
    chans, _, _ = leaves(H, W, k, taps)
    for ch in chans:
        f = np.real(np.fft.ifft2(ch["F"] * X))
        if k == 1:
            r = np.arange(H)[:, None]
            c = 2 * np.arange(W // 2)[None, :] + ((r + ch["o"][0] + ch["o"][1]) & 1)
            out.append(f[r, c].ravel())
        else:
            R, C = (2 ** (k - 1), 2) if ch["T"] == "c" else (2, 2 ** (k - 1))
            out.append(f[ch["o"][0] % R::R, ch["o"][1] % C::C].ravel())
    return np.concatenate(out)


def wedge_mask(ch, k, wr, wc):
    """Ideal wedge of a leaf: F_c leaves cover slopes w_r/w_c in [i/2^m, (i+1)/2^m] inside
    |w_c| >= |w_r|; F_r leaves the same for w_c/w_r inside |w_r| > |w_c| (m = k - 2)."""
    if k == 1:
        return (np.abs(wc) >= np.abs(wr)) if ch["T"] == "c" else (np.abs(wr) > np.abs(wc))
    m, i = k - 2, ch["i"]
    with np.errstate(divide="ignore", invalid="ignore"):
        if ch["T"] == "c":
            s = wr / wc
            return (np.abs(wc) >= np.abs(wr)) & (s >= i / 2 ** m) & (s < (i + 1) / 2 ** m)
        t = wc / wr
        return (np.abs(wr) > np.abs(wc)) & (t >= i / 2 ** m) & (t < (i + 1) / 2 ** m)


def wedge_fractions(k, N=128, taps=None):
    """Per leaf: fraction of its equivalent filter's energy, over the high-frequency
    annulus pi/2 < |w| (where LP details live), that falls inside its own wedge."""
    chans, wr, wc = leaves(N, N, k, taps)
    ann = np.hypot(wr, wc) > np.pi / 2
    fr = []
    for ch in chans:
        E = np.abs(ch["F"]) ** 2 * ann
        fr.append(float((E * wedge_mask(ch, k, wr, wc)).sum() / E.sum()))
    return fr
