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
  5. mirror window (mirror=True): a node whose window split along direction
     d is scanned once more in a window of half-width (w + 1) // 2 centred on
     the cell of d reflected about the principal axes of F (mirror_angles:
     an isotropic W takes the same values on both lines, so every local
     minimum over the angles has a twin of the same value there), with the
     same re-centring; the node takes the lower of the two values (the lower
     global direction index on equal values) and falls back if the mirror
     window's best still lies on its border.  It is skipped when the mirror
     window lies inside the last main window;
  6. the split and the recursion are those of the plain method.
Every integer decision comes with its margin: the distance of the scaled
angles to a rounding boundary (in cells), the scan's certified margin,
|gap - gap_tol| relative to gap_tol, and |V_mirror - V| for the mirror's
choice.
"""
from __future__ import annotations

import math

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


def principal_angles(F):
    """Angles phi1, phi2 of the first left and right singular vectors of the
    2 x 2 matrix F (the eigenvectors of F F^T and F^T F with the larger
    eigenvalue): for a symmetric [[A, B], [B, C]] that eigenvector lies at
    0.5 atan2(2B, A - C).  (0, 0) when the eigenvalues coincide."""
    f00, f01, f10, f11 = (float(x) for x in np.asarray(F, dtype=np.float64).reshape(4))
    p1 = 0.5 * math.atan2(2.0 * (f00 * f10 + f01 * f11),
                          (f00 * f00 + f01 * f01) - (f10 * f10 + f11 * f11))
    p2 = 0.5 * math.atan2(2.0 * (f00 * f01 + f10 * f11),
                          (f00 * f00 + f10 * f10) - (f01 * f01 + f11 * f11))
    return p1, p2


def mirror_angles(F, ta, tb):
    """The rank-one direction a(ta) (x) b(tb) reflected about the principal
    axes of F.  With F = Q1 S Q2^T and the reflections M1 = Q1 diag(1, -1)
    Q1^T, M2 = Q2 diag(1, -1) Q2^T, M1 F M2 = F, so
    M1 (F + t a (x) b) M2 = F + t (M1 a) (x) (M2 b): both lines have the same
    ||.||^2 and det at every t, hence the same values of an isotropic W
    (Sec. 2: W depends on F through I1 and J) and the same hull.  M1 maps the
    angle ta to 2 phi1 - ta, M2 maps tb to 2 phi2 - tb (angles mod pi)."""
    p1, p2 = principal_angles(F)
    return 2.0 * p1 - ta, 2.0 * p2 - tb


def mirror_cell(F, gd, Na, Nb):
    """Grid cell nearest to the mirror of direction gd = ia * Nb + ib of the
    angle grid (theta = pi i / N) and the distance of the scaled angles to a
    rounding boundary (in cells), the margin of that integer decision."""
    ia, ib = gd // Nb, gd % Nb
    p1, p2 = principal_angles(F)
    ua = 2.0 * p1 * Na / math.pi - ia
    ub = 2.0 * p2 * Nb / math.pi - ib
    ma = int(math.floor(ua + 0.5)) % Na
    mb = int(math.floor(ub + 0.5)) % Nb
    dist = min(abs(ua + 0.5 - round(ua + 0.5)), abs(ub + 0.5 - round(ub + 0.5)))
    return (ma, mb), dist


def propose_convexify(orc, mat, Na, Nb, L, t_half, K, w, gap_tol, flat, mean, std, F, beta,
                      one_sided=False, recentre=0, mirror=False):
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

            def search(ca, cb, hw, gap_test):
                """Window scans from centre (ca, cb), half-width hw, re-centred
                on a border minimum while the gap test passes."""
                margin = np.inf
                for moves in range(recentre + 1):
                    idx = window_indices(ca, cb, hw, Na, Nb)
                    order = np.argsort(idx, kind="stable")  # lowest global index wins ties
                    sc = orc.Scan(dirs_all[idx[order]], L, t_half, 1)
                    info = orc.scan_node(mat, sc, Fi, b)
                    margin = min(margin, info["margin"])
                    gd = int(idx[order][info["dir"]])
                    lam = info["m_minus"] != m0
                    V = info["h"] if lam else rec["w"]
                    border = lam and (abs(_offset(gd // Nb, ca, Na)) >= hw or
                                      abs(_offset(gd % Nb, cb, Nb)) >= hw)
                    gap = ((V - E_pred) if one_sided else abs(E_pred - V)) / (1e-8 + abs(V))
                    ok = gap <= gap_tol or not gap_test
                    if not (border and ok) or moves == recentre:
                        break
                    ca, cb = gd // Nb, gd % Nb  # re-centre on the border minimum
                return info, gd, lam, V, border, gap, moves, margin, (ca, cb)

            info, gd, lam, V, border, gap, moves, window_margin, (ca, cb) = search(ia, ib, w, True)
            rec.update(gap=gap, window_margin=window_margin, window_dir=gd, window_lam=lam, V=V,
                       recentred=moves, last_center=(ca, cb))
            if mirror and lam and not (border or not gap <= gap_tol):
                mc, mdist = mirror_cell(Fi, gd, Na, Nb)
                wm = (w + 1) // 2
                inside = (abs(_offset(mc[0], ca, Na)) + wm <= w and
                          abs(_offset(mc[1], cb, Nb)) + wm <= w)
                rec.update(mirror_center=mc, mirror_center_margin=mdist, mirror_inside=inside)
                if not inside:
                    info2, gd2, lam2, V2, border2, _, moves2, m2, _ = search(mc[0], mc[1], wm, False)
                    rec.update(mirror_dir=gd2, mirror_recentred=moves2, mirror_gap=abs(V2 - V),
                               window_margin=min(window_margin, m2), mirror_won=False)
                    if border2:
                        border = True
                    elif lam2 and (V2 < V or (V2 == V and gd2 < gd)):
                        info, gd, V = info2, gd2, V2
                        rec["mirror_won"] = True
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
