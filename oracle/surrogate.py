"""Oracle of the surrogate-proposed convexification (test infrastructure only).

TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and bench.py's CPU
baseline may use this module.

Per tree node, top-down as the plain method (Eq. 3.3 per point):
  1. the network (oracle.mlp, with the BF16 rounding points of a tensor-core
     implementation) proposes angles, xi and the jump; the angles' nearest
     cell (ia, ib) of the Na x Nb grid centres a window of (2w + 1)^2
     directions (indices wrap);
  2. the line scan (Sec. 4, the oracle's own C scan) runs over the window's
     directions only;
  3. if the window's best direction lies on the window border (and the energy
     gap test below passes), the window is moved to be centred on that
     direction's cell and scanned again, at most ``recentre`` times (a local
     descent over the angle grid; recentre = 0 does not move it);
  4. the node falls back to the scan of all directions if the window's best
     direction still lies on the window border or the energy gap
     |E_pred - V| / (1e-8 + |V|) exceeds gap_tol, with V the window's node
     value and E_pred = xi W(F+) + (1 - xi) W(F-) of the proposed laminate
     (one_sided: (V - E_pred) / (1e-8 + |V|), only a better proposal counts);
  5. the split and the recursion are those of the plain method.
Every integer decision comes with its margin: the distance of the scaled
angles to a rounding boundary (in cells), the scan's certified margin, and
|gap - gap_tol| relative to gap_tol.
"""
from __future__ import annotations

import numpy as np

from . import mlp

FALLBACK = 32


def window_indices(ia, ib, w, Na, Nb):
    """Global direction indices of the window, in the scan's order."""
    out = []
    for da in range(-w, w + 1):
        for db in range(-w, w + 1):
            out.append(((ia + da) % Na) * Nb + ((ib + db) % Nb))
    return np.array(out)


def _offset(i, c, N):
    d = (i - c) % N
    return d - N if d > N // 2 else d


def propose_convexify(orc, mat, Na, Nb, L, t_half, K, w, gap_tol, flat, mean, std, F, beta,
                      one_sided=False, recentre=0):
    """Returns (W_R, P, nodes) with nodes[p] = {heap index: record}."""
    dirs_all = orc.angle_directions(Na, Nb)
    full = orc.Scan(dirs_all, L, t_half, 1)
    m0 = (L - 1) // 2
    hstep = 2.0 * t_half / (L - 1)
    F = np.asarray(F, dtype=np.float64).reshape(-1, 4)
    n = F.shape[0]
    WR = np.zeros(n)
    P = np.zeros((n, 4))
    trees = []
    for p in range(n):
        b = float(beta[p])
        nodes = {}

        def build(i, Fi, weight, left):
            rec = dict(F=Fi.copy(), w=orc.energy(mat, Fi, b), weight=weight, flags=0, dir=-1)
            nodes[i] = rec
            if left == 0:
                return
            out, _ = mlp.forward(flat, mlp.features(Fi, b), mean, std, bf=True)
            ia, ib, xi_p, Fp, Fm, dist = mlp.decode(out, Fi, Na, Nb)
            ia, ib = int(ia[0]), int(ib[0])
            E_pred = xi_p[0] * orc.energy(mat, Fp[0], b) + (1 - xi_p[0]) * orc.energy(mat, Fm[0], b)
            rec.update(center=(ia, ib), center_margin=float(dist[0]), E_pred=E_pred)
            ca, cb = ia, ib
            window_margin = np.inf
            for moves in range(recentre + 1):
                idx = window_indices(ca, cb, w, Na, Nb)
                order = np.argsort(idx, kind="stable")  # lowest global index wins ties
                sc = orc.Scan(dirs_all[idx[order]], L, t_half, 1)
                info = orc.scan_node(mat, sc, Fi, b)
                window_margin = min(window_margin, info["margin"])
                gd = int(idx[order][info["dir"]])
                lam = info["m_minus"] != m0
                V = info["h"] if lam else rec["w"]
                border = lam and (abs(_offset(gd // Nb, ca, Na)) >= w or
                                  abs(_offset(gd % Nb, cb, Nb)) >= w)
                gap = ((V - E_pred) if one_sided else abs(E_pred - V)) / (1e-8 + abs(V))
                if not (border and gap <= gap_tol) or moves == recentre:
                    break
                ca, cb = gd // Nb, gd % Nb  # re-centre on the border minimum
            rec.update(gap=gap, window_margin=window_margin, window_dir=gd, window_lam=lam, V=V,
                       recentred=moves, last_center=(ca, cb))
            if border or not gap <= gap_tol:
                info = orc.scan_node(mat, full, Fi, b)
                gd = info["dir"]
                lam = info["m_minus"] != m0
                rec["flags"] |= FALLBACK
            rec["margin"] = info["margin"]
            rec["flags"] |= orc.SCANNED
            if not lam:
                return
            rec["flags"] |= orc.LAMINATED
            rec.update(dir=gd, m_minus=info["m_minus"], m_plus=info["m_plus"], h=info["h"])
            R = orc.rank_one(dirs_all[gd])
            tm = (info["m_minus"] - m0) * hstep
            tp = (info["m_plus"] - m0) * hstep
            xi = (m0 - info["m_minus"]) / (info["m_plus"] - info["m_minus"])
            rec["xi"] = xi
            build(2 * i + 1, Fi + tm * R, weight * (1 - xi), left - 1)
            build(2 * i + 2, Fi + tp * R, weight * xi, left - 1)

        build(0, F[p], 1.0, K)
        W = 0.0
        Pp = np.zeros(4)
        for rec in nodes.values():
            if rec["flags"] & orc.LAMINATED:
                continue
            W += rec["weight"] * orc.energy(mat, rec["F"], b)
            Pp += rec["weight"] * orc.stress(mat, rec["F"], b)
        WR[p] = W
        P[p] = Pp
        trees.append(nodes)
    return WR, P, trees
