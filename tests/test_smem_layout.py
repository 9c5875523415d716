"""Shared-memory bank model of the P = 8 element stages (host-side check).

The element kernels keep one element's fields in shared memory and walk
them along lines of Gauss points (sum factorisation of eq.
ProdTensorialHexaedro).  For P = 8 the y- and z-line stages give each warp
one slab of lines across the three components, and the field pitches are
padded, so that every warp access lands in 32 distinct banks.  This test
restates the pitches and thread-to-line maps of the kernel header and counts
shared-memory wavefronts per element with the 32-bank model, so a change of
either side that brings conflicts back fails here, without a GPU."""
import collections
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2104_13466_gb300", "csrc", "elem_kernels.cuh")

P = 8
n, Q = P + 1, P + 2
NT = (3 * Q * Q + 31) // 32 * 32
XQ, XN = Q | 1, n | 1
SPQ = SP2 = Q * XQ + 1
FQ = Q * SPQ
SX, SA1 = n * n * XN, n * n * XQ
SA2 = (n * SP2 + 31 - Q) // 32 * 32 + Q


def _wavefronts(addrs):
    banks = collections.defaultdict(set)
    for a in addrs:
        banks[a % 32].add(a)
    return max(len(s) for s in banks.values())


def _packed(ni, nj):
    lines = [(c, i, j) for c in range(3) for i in range(ni) for j in range(nj)]
    return [lines[k:k + 32] for k in range(0, len(lines), 32)]


def _slab(nslab, m):
    # warp w: slab w; lane c * m + j: (component c, index j)
    return [[(c, w, j) for c in range(3) for j in range(m)] for w in range(nslab)]


def _count(warps, base, nacc, stride):
    tot = ideal = 0
    for w in warps:
        for a in range(nacc):
            tot += _wavefronts([base(*x) + a * stride for x in w])
            ideal += 1
    return tot, ideal


def _stages():
    rows = _packed(n, n)                                    # (c, r, q)
    cols = [[(c, r, qx) for (c, qx, r) in w] for w in _slab(Q, n)]   # warp qx, lanes (c, r)
    zc = _slab(Q, Q)                                        # warp qy, lanes (c, qx)
    xl = [[(c, qz, qy) for (c, qy, qz) in w] for w in _slab(Q, Q)]   # warp qy, lanes (c, qz)
    yl = _slab(Q, Q)                                        # warp qz, lanes (c, qx)
    out = {
        "F1 X": _count(rows, lambda c, r, q: c * SX + (r * n + q) * XN, n, 1),
        "F1 A1": _count(rows, lambda c, r, q: c * SA1 + (r * n + q) * XQ, Q, 1),
        "F2 A1": _count(cols, lambda c, r, qx: c * SA1 + r * n * XQ + qx, n, XQ),
        "F2 A2": _count(cols, lambda c, r, qx: c * SA2 + r * SP2 + qx, Q, XQ),
        "F3 A2": _count(zc, lambda c, qy, qx: c * SA2 + qy * XQ + qx, n, SP2),
        "F3 U": _count(zc, lambda c, qy, qx: c * FQ + qy * XQ + qx, Q, SPQ),
        "D x": _count(xl, lambda c, qz, qy: c * FQ + qz * SPQ + qy * XQ, Q, 1),
        "D y": _count(yl, lambda c, qz, qx: c * FQ + qz * SPQ + qx, Q, XQ),
    }
    # pointwise walk: pass p takes rows 3p .. 3p + 2 of the Q^2 rows (qz, qy)
    rows = [(qz, qy) for qz in range(Q) for qy in range(Q)]
    pw = [[qz * SPQ + qy * XQ + qx for (qz, qy) in rows[3 * p:3 * p + 3] for qx in range(Q)]
          for p in range((Q * Q + 2) // 3)]
    out["pointwise"] = (sum(_wavefronts(g) for g in pw), len(pw))
    return out


def test_header_states_the_modelled_pitches():
    src = open(HEADER).read()
    for pat in (r"SPQ = Q \* XQ \+ \(SLAB \? 1 : 0\)", r"FQ = Q \* SPQ", r"SP2 = Q \* XQ \+ \(SLAB \? 1 : 0\)",
                r"SA2 = SLAB \? \(n \* SP2 \+ 31 - Q\) / 32 \* 32 \+ Q", r"on = slab_line<P>\(t, n, &c, &qx, &r\)",
                r"on = slab_line<P>\(t, Q, &c, &qy, &qx\)", r"on = slab_line<P>\(t, Q, &c, &qy, &qz\)",
                r"on = slab_line<P>\(t, Q, &c, &qz, &qx\)", r"WALK = G::SLAB \? \(Q \* Q \+ 2\) / 3 \* 32 : Q3"):
        assert re.search(pat, src), pat
    assert NT // 32 >= Q and 3 * Q <= 32          # the slab maps apply at P = 8


def test_every_p8_stage_access_is_conflict_free():
    for name, (tot, ideal) in _stages().items():
        if name == "pointwise":
            # a pass whose three rows straddle a z-slab meets its own first
            # bank again once: at most one two-way conflict per slab boundary
            assert tot <= ideal + Q - 1, (tot, ideal)
        else:
            assert tot == ideal, (name, tot, ideal)


def test_slab_fields_fit_four_float32_ctas_per_sm():
    words = 12 * FQ
    assert 3 * SA2 <= 3 * FQ and 3 * SA1 <= 3 * FQ and 3 * SX <= 3 * FQ
    assert 4 * (4 * words + 272 + 1024) <= 233472   # 228 KB of shared memory per SM
    # the pointwise walk: 34 warp passes of 30 lanes for the 1000 Gauss points
    assert (Q * Q + 2) // 3 == 34
