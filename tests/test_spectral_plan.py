"""Host-logic test of the spectral control's line transforms (Sec. 3.2): the level plan and the
index scheme the kernels use (csrc/lb_spectral_fft.cuh), restated in numpy and run on the CPU
for every grid edge 4 ... 4096. The largest radix is read from the header, so a change of the
plan there is tested here. Checks: the levels reproduce the DFT (forward and inverse), every
shared-memory index stays inside the padded line, every twiddle index inside the table, the
last level's outputs are each element once, and the column kernels' forward output order is a
permutation of the inverse's input order (the registers a thread holds)."""
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2106_12929_gb300", "csrc", "lb_spectral_fft.cuh")


def max_b0() -> int:
    m = re.search(r"constexpr int kMaxB0 = (\d+);", open(HDR).read())
    assert m, "kMaxB0 not found in the header"
    return int(m.group(1))


def plan(L: int, mb: int):
    N = 1 << L
    b0 = L if L <= mb else ((L + 1) // 2 if L <= 2 * mb else mb)
    rest = L - b0
    nlev = 1 if rest == 0 else (2 if rest <= b0 else 3)
    b1 = 0 if nlev == 1 else (rest if nlev == 2 else (rest + 1) // 2)
    b2 = rest - b1 if nlev == 3 else 0
    P = 1 << b0
    M, R1, R2 = N // P, 1 << b1, 1 << b2
    RL = P if nlev == 1 else (R1 if nlev == 2 else R2)
    tw2 = (R1 - 1) * P if nlev >= 2 else 0
    twn = tw2 + ((R2 - 1) * P * R1 if nlev == 3 else 0)
    base = N + N // P
    LS = base + (20 - base % 16) % 16
    return dict(N=N, b0=b0, nlev=nlev, bits=[b0, b1, b2][:nlev], P=P, M=M, R1=R1, R2=R2, RL=RL, SUBL=P // RL,
                TW2=tw2, TWN=twn, LS=LS)


def table(p):
    """The level twiddles exp(-2 pi i m r / (Ns R)) in the kernels' layout."""
    tw = np.zeros(max(p["TWN"], 1), complex)
    for e in range(p["TWN"]):
        if e < p["TW2"]:
            ns, rad, r, m = p["P"], p["R1"], e // p["P"] + 1, e % p["P"]
        else:
            ns = p["P"] * p["R1"]
            rad, r, m = p["R2"], (e - p["TW2"]) // ns + 1, (e - p["TW2"]) % ns
        tw[e] = np.exp(-2j * np.pi * m * r / (ns * rad))
    return tw


def line_transform(x, p, inv=False):
    """The kernels' steps for one line: per thread t the registers a[0..P), the shared line z."""
    N, P, M, b0 = p["N"], p["P"], p["M"], p["b0"]
    sgn = 1 if inv else -1
    tw = table(p)
    if inv:
        tw = np.conj(tw)
    pad = lambda q: q + (q >> b0)  # noqa: E731
    z = np.full(p["LS"], np.nan, complex)
    regs = [np.array([x[t + r * M] for r in range(P)]) for t in range(M)]

    def dft(v):
        R = len(v)
        return np.array([sum(v[r] * np.exp(sgn * 2j * np.pi * r * k / R) for r in range(R)) for k in range(R)])

    regs = [dft(a) for a in regs]
    if p["nlev"] >= 2:
        for t in range(M):
            for k in range(P):
                q = pad(t * P + k)
                assert q < p["LS"]
                z[q] = regs[t][k]
    ns = P
    for lev in range(1, p["nlev"]):
        rad = 1 << p["bits"][lev]
        sub, two = P // rad, (0 if lev == 1 else p["TW2"])
        last = lev == p["nlev"] - 1
        new = []
        for t in range(M):
            a = np.zeros(P, complex)
            for s in range(sub):
                j = t + M * s
                m = j & (ns - 1)
                for r in range(rad):
                    q = pad(j + r * (N // rad))
                    assert q < p["LS"]
                    a[s * rad + r] = z[q]
                for r in range(1, rad):
                    e = two + (r - 1) * ns + m
                    assert e < p["TWN"]
                    a[s * rad + r] *= tw[e]
                a[s * rad:(s + 1) * rad] = dft(a[s * rad:(s + 1) * rad])
            new.append(a)
        if not last:
            z[:] = np.nan
            for t in range(M):
                for s in range(sub):
                    j = t + M * s
                    m = j & (ns - 1)
                    d = (j // ns) * ns * rad + m
                    for k in range(rad):
                        q = pad(d + k * ns)
                        assert q < p["LS"]
                        z[q] = new[t][s * rad + k]
        regs = new
        ns *= rad
    out = np.full(N, np.nan, complex)
    for t in range(M):
        for s in range(p["SUBL"]):
            for k in range(p["RL"]):
                i = t + M * s + k * (N // p["RL"])
                assert np.isnan(out[i])  # each element once
                out[i] = regs[t][s * p["RL"] + k]
    return out


@pytest.mark.parametrize("L", list(range(2, 13)))
def test_line_transform_plan_reproduces_the_dft(L):
    p = plan(L, max_b0())
    assert p["P"] <= 32 and p["nlev"] <= 3 and sum(p["bits"]) == L
    assert max(p["bits"]) == p["b0"]  # every later level fits the P values of a thread
    rng = np.random.default_rng(L)
    x = rng.standard_normal(p["N"]) + 1j * rng.standard_normal(p["N"])
    assert np.allclose(line_transform(x, p), np.fft.fft(x), rtol=0, atol=1e-9 * p["N"])
    assert np.allclose(line_transform(x, p, inv=True), np.fft.ifft(x) * p["N"], rtol=0, atol=1e-9 * p["N"])


@pytest.mark.parametrize("L", list(range(2, 13)))
def test_forward_output_order_is_the_inverse_input_order(L):
    """A thread's forward outputs t + M s + k N / RL are its inverse inputs t + r M: the column
    kernels could keep a column in registers between the two transforms."""
    p = plan(L, max_b0())
    N, M = p["N"], p["M"]
    for t in range(M):
        outs = sorted(t + M * s + k * (N // p["RL"]) for s in range(p["SUBL"]) for k in range(p["RL"]))
        assert outs == sorted(t + r * M for r in range(p["P"]))
