"""Adaptive 3:1 tree mesh for the ADER-DG oracle (Sec. 3 AMR criterion,
Sec. 4.2 runs with two refinement levels; cell sizes 1000/9, 1000/27,
1000/81 m in the paper).  TEST INFRASTRUCTURE (see oracle/__init__.py).

Readings (the paper gives the criterion, Eqs. 6-7, and "subcells are
coarsened only if all subcells belonging to the coarse cell are marked for
coarsening", but not the mesh operations):

A1  refinement splits a cell into 3 x 3 children; the children's nodal
    values are the parent polynomial evaluated at their nodes (exact);
A2  coarsening replaces 9 sibling leaves, all flagged -1, by their parent;
    the parent's nodal values are the L2 projection of the 9 children by
    Gauss-Legendre quadrature on each child (exact, conserves every
    integral);
A3  neighbouring leaves differ by at most one level; refinement wins
    (neighbours of a refined cell that would be two levels coarser are
    refined too; a sibling group whose parent would touch a leaf two levels
    finer is kept);
A4  hanging faces (one coarse face against three fine faces): the fine side
    sees the coarse trace evaluated on its third of the face; the coarse side
    receives the L2 restriction of the three fine numerical fluxes, which
    keeps the scheme conservative; the Rusanov penalty uses the fine cell size
    on both sides;
A5  leaves are ordered by (level, iy, ix) after every adaptation.

L1  local time stepping (step_lts, not in the paper): a leaf of level l steps
    with dt 3^(L-l); at a hanging face the fine side sees the coarse
    predictor's trace averaged over the third of the coarse step its own step
    covers, and the coarse side receives the time average of the fine
    numerical fluxes of its three sub-steps (restricted per spatial third).

Pins: tests/test_oracle_amr.py (restrict(prolong(u)) = u, conservation of
all integrals over steps with hanging faces and across adaptation, a mesh
refined everywhere reproduces the uniform fine run, the balance rule);
tests/test_oracle_lts.py (local time stepping).
"""
import itertools

import torch

from . import DTYPE
from .aderdg import Mesh, Solver
from .basis import lagrange_values
from . import physics as ph


class _LevelView(Solver):
    """Oracle Solver restricted to the leaves of one level (cell-local work)."""

    def __init__(self, amr, level, leaves):
        self.P = amr.P
        self.b = amr.b
        hx, hy = amr.h(level)
        self.m = Mesh(nx=1, ny=1, Lx=hx, Ly=hy)
        n = self.b.n
        xi = self.b.xi
        ix = torch.tensor([c[1] for c in leaves], dtype=DTYPE)
        iy = torch.tensor([c[2] for c in leaves], dtype=DTYPE)
        xs = amr.x0 + (ix[:, None] + xi[None, :]) * hx          # [c, i]
        ys = amr.y0 + (iy[:, None] + xi[None, :]) * hy          # [c, j]
        self.X = xs[:, None, :].expand(-1, n, n)
        self.Y = ys[:, :, None].expand(-1, n, n)
        self.Kw = self.b.K1inv * self.b.w[None, :]


class AmrSolver:
    """Plain FP64 ADER-DG on a 3:1 adaptive tree of square-grid cells."""

    def __init__(self, base_nx, base_ny, params, Lx, Ly, x0=0.0, y0=0.0, bc="wall", max_level=2):
        self.nx0, self.ny0 = base_nx, base_ny
        self.Lx, self.Ly, self.x0, self.y0 = Lx, Ly, x0, y0
        self.P = params
        self.bc = bc
        self.max_level = max_level
        self.ref = Solver(Mesh(base_nx, base_ny, x0=x0, y0=y0, Lx=Lx, Ly=Ly), params)
        self.b = self.ref.b
        n = self.b.n
        xi = self.b.xi
        # 1D prolongation P[a][m][q] = phi_q((a + xi_m) / 3)
        self.Pro = torch.stack([lagrange_values(xi, (a + xi) / 3.0) for a in range(3)])
        self.leaves = [(0, ix, iy) for iy in range(base_ny) for ix in range(base_nx)]
        self._index()

    # -------------------------------------------------------------- geometry
    def h(self, level):
        return self.Lx / (self.nx0 * 3 ** level), self.Ly / (self.ny0 * 3 ** level)

    def _index(self):
        self.leaves.sort(key=lambda c: (c[0], c[2], c[1]))   # reading A5: (level, iy, ix)
        self.pos = {c: k for k, c in enumerate(self.leaves)}

    def extent(self, level):
        return self.nx0 * 3 ** level, self.ny0 * 3 ** level

    def neighbour(self, leaf, face):
        """('conf', k) | ('coarse', k, s) | ('fine', [k0, k1, k2]) | ('wall',)."""
        lv, ix, iy = leaf
        NX, NY = self.extent(lv)
        dx, dy = {"E": (1, 0), "W": (-1, 0), "N": (0, 1), "S": (0, -1)}[face]
        jx, jy = ix + dx, iy + dy
        if not (0 <= jx < NX and 0 <= jy < NY):
            if self.bc == "wall":
                return ("wall",)
            jx, jy = jx % NX, jy % NY
        if (lv, jx, jy) in self.pos:
            return ("conf", self.pos[(lv, jx, jy)])
        if lv > 0 and (lv - 1, jx // 3, jy // 3) in self.pos:
            s = iy % 3 if face in ("E", "W") else ix % 3
            return ("coarse", self.pos[(lv - 1, jx // 3, jy // 3)], s)
        kids = []
        for s in range(3):
            if face == "E":
                c = (lv + 1, 3 * jx, 3 * iy + s)
            elif face == "W":
                c = (lv + 1, 3 * jx + 2, 3 * iy + s)
            elif face == "N":
                c = (lv + 1, 3 * ix + s, 3 * jy)
            else:
                c = (lv + 1, 3 * ix + s, 3 * jy + 2)
            kids.append(self.pos[c])  # KeyError here means an unbalanced tree
        return ("fine", kids)

    def levels(self):
        return sorted({c[0] for c in self.leaves})

    def level_views(self):
        out = []
        for lv in self.levels():
            idx = [k for k, c in enumerate(self.leaves) if c[0] == lv]
            out.append((lv, torch.tensor(idx), _LevelView(self, lv, [self.leaves[k] for k in idx])))
        return out

    def node_coords(self):
        n = self.b.n
        X = torch.empty(len(self.leaves), n, n, dtype=DTYPE)
        Y = torch.empty_like(X)
        for lv, idx, view in self.level_views():
            X[idx], Y[idx] = view.X, view.Y
        return X, Y

    # -------------------------------------------------------------- scheme
    def step(self, u, dt, t=0.0):
        P = self.P
        b = self.b
        n = b.n
        C = len(self.leaves)
        tavg = {k: torch.empty(C, 4, n, n, dtype=DTYPE) for k in ("qbar", "Fbar", "Gbar", "Sbar", "qxbar", "qybar")}
        for lv, idx, view in self.level_views():
            _, ta = view.predictor(u[idx], dt, t)
            for k in tavg:
                tavg[k][idx] = ta[k]
        tr = self.ref.face_traces(tavg)          # cell-local extrapolation, any h
        Fst = {f: torch.empty(C, 4, n, dtype=DTYPE) for f in "EWNS"}
        nrm = {"E": (1.0, 0.0), "W": (1.0, 0.0), "N": (0.0, 1.0), "S": (0.0, 1.0)}
        opp = {"E": "W", "W": "E", "N": "S", "S": "N"}
        for k, leaf in enumerate(self.leaves):
            lv, ix, iy = leaf
            hx, hy = self.h(lv)
            for f in "EWNS":
                xf = f in "EW"
                hn = hx if xf else hy
                own_minus = f in "EN"           # own cell on the - side of the face
                z = self._face_z(leaf, f)
                nb = self.neighbour(leaf, f)
                own = {key: tr[f][key][k:k + 1] for key in ("q", "f", "qx", "qy")}
                if nb[0] == "wall":
                    normal = {"E": (1.0, 0.0), "W": (-1.0, 0.0), "N": (0.0, 1.0), "S": (0.0, -1.0)}[f]
                    gq, gf = self.ref._ghost(own, normal, z)
                    F = self._riemann(own["q"], own["f"], gq, gf, z, own_minus, nrm[f], hn)
                elif nb[0] == "conf":
                    o = nb[1]
                    F = self._riemann(own["q"], own["f"], tr[opp[f]]["q"][o:o + 1], tr[opp[f]]["f"][o:o + 1],
                                      z, own_minus, nrm[f], hn)
                elif nb[0] == "coarse":
                    o, s = nb[1], nb[2]
                    cq = self._prolong_face(tr[opp[f]]["q"][o:o + 1], s)
                    cf = self._prolong_face(tr[opp[f]]["f"][o:o + 1], s)
                    F = self._riemann(own["q"], own["f"], cq, cf, z, own_minus, nrm[f], hn)
                else:  # three finer neighbours: restrict their fluxes
                    hf = hn / 3.0
                    subs = []
                    for s, o in enumerate(nb[1]):
                        cq = self._prolong_face(own["q"], s)
                        cf = self._prolong_face(own["f"], s)
                        zf = self._face_z(self.leaves[o], opp[f])
                        subs.append(self._riemann(tr[opp[f]]["q"][o:o + 1], tr[opp[f]]["f"][o:o + 1], cq, cf,
                                                  zf, not own_minus, nrm[f], hf))
                    F = self._restrict_face(subs)
                Fst[f][k] = F[0]
        # update with each leaf's cell size
        w, p0, p1 = b.w, b.phi0, b.phi1
        Vx = (w[:, None] * b.D) / w[None, :]
        out = torch.empty_like(u)
        for lv, idx, view in self.level_views():
            hx, hy = self.h(lv)
            vol = (torch.einsum("pi,cvjp->cvji", Vx, tavg["Fbar"][idx]) / hx
                   + torch.einsum("pj,cvpi->cvji", Vx, tavg["Gbar"][idx]) / hy)
            FE, FW, GN, GS = Fst["E"][idx], Fst["W"][idx], Fst["N"][idx], Fst["S"][idx]
            face = ((p1[None, None, None, :] * FE[:, :, :, None] - p0[None, None, None, :] * FW[:, :, :, None])
                    / (hx * w[None, None, None, :])
                    + (p1[None, None, :, None] * GN[:, :, None, :] - p0[None, None, :, None] * GS[:, :, None, :])
                    / (hy * w[None, None, :, None]))
            out[idx] = u[idx] + dt * (vol - face + tavg["Sbar"][idx])
        return out

    # -------------------------------------------------------------- local time stepping
    def time_thirds(self):
        """W[s][k]: average over the third s of the step of the nodal time
        interpolant's basis function k, sum_m w_m phi_k((s + xi_m)/3) (n-point
        Gauss-Legendre on the third, exact for the degree-N interpolant)."""
        xi, w = self.b.xi, self.b.w
        return torch.stack([torch.einsum("m,mk->k", w, lagrange_values(xi, (s + xi) / 3.0)) for s in range(3)])

    def step_lts(self, u, dt, t=0.0):
        """One cycle of local time stepping (reading L1): leaves of level l
        advance by dt 3^(L-l), L the finest level present, in 3^(L-l0) steps
        of the finest level (l0 the coarsest).  A level's step is its
        predictor over its whole step, then three steps of the next finer
        level, then its corrector.  Between levels: the finer side of a
        hanging face takes the coarse predictor's trace averaged over the
        third of the coarse step that its own step covers (the W weights of
        time_thirds); the coarse side receives, per spatial third of the
        face, the average of the three fine numerical fluxes of its three
        sub-steps, then their L2 restriction -- conservative, because it is
        the fine flux integral itself.  On a tree with one level this is the
        global step.  Returns (state, cycle length)."""
        levels = self.levels()
        L, l0 = max(levels), min(levels)
        self._lts_u = u.clone()
        self._lts_sub = {}
        self._lts_acc = {}
        self._lts_W = self.time_thirds()
        self._lts_level(l0, t, dt, L, 0)
        u_new = self._lts_u
        del self._lts_u, self._lts_sub, self._lts_acc, self._lts_W
        return u_new, dt * 3 ** (L - l0)

    def _lts_level(self, lv, t, dt, L, kstep):
        b = self.b
        n = b.n
        dtl = dt * 3 ** (L - lv)
        idx = [k for k, c in enumerate(self.leaves) if c[0] == lv]
        loc = {k: a for a, k in enumerate(idx)}
        view = _LevelView(self, lv, [self.leaves[k] for k in idx])
        q, tavg = view.predictor(self._lts_u[idx], dtl, t)
        tr = self.ref.face_traces(tavg)
        finer = lv + 1 in self.levels()
        if finer:
            if self.P.source != "none":
                Sman = torch.stack([view.manufactured(t + float(b.xi[k]) * dtl) for k in range(n)], 1)
            else:
                Sman = None
            F, G, S, qx, qy = view.evaluate(q, Sman)
            self._lts_sub[lv] = []
            for s in range(3):
                Ws = self._lts_W[s]
                avg = lambda a: torch.einsum("k,ck...->c...", Ws, a)
                self._lts_sub[lv].append(self.ref.face_traces(dict(qbar=avg(q), Fbar=avg(F), Gbar=avg(G),
                                                                   qxbar=avg(qx), qybar=avg(qy))))
            for k in idx:
                for f in "EWNS":
                    if self.neighbour(self.leaves[k], f)[0] == "fine":
                        self._lts_acc[(k, f)] = [torch.zeros(1, 4, n, dtype=DTYPE) for _ in range(3)]
            for ks in range(3):
                self._lts_level(lv + 1, t + ks * dtl / 3.0, dt, L, ks)
        # corrector of this level
        nrm = {"E": (1.0, 0.0), "W": (1.0, 0.0), "N": (0.0, 1.0), "S": (0.0, 1.0)}
        opp = {"E": "W", "W": "E", "N": "S", "S": "N"}
        Fst = {f: torch.empty(len(idx), 4, n, dtype=DTYPE) for f in "EWNS"}
        for a, k in enumerate(idx):
            leaf = self.leaves[k]
            hx, hy = self.h(lv)
            for f in "EWNS":
                xf = f in "EW"
                hn = hx if xf else hy
                own_minus = f in "EN"
                z = self._face_z(leaf, f)
                nb = self.neighbour(leaf, f)
                own = {key: tr[f][key][a:a + 1] for key in ("q", "f", "qx", "qy")}
                if nb[0] == "wall":
                    normal = {"E": (1.0, 0.0), "W": (-1.0, 0.0), "N": (0.0, 1.0), "S": (0.0, -1.0)}[f]
                    gq, gf = self.ref._ghost(own, normal, z)
                    Fv = self._riemann(own["q"], own["f"], gq, gf, z, own_minus, nrm[f], hn)
                elif nb[0] == "conf":
                    o = loc[nb[1]]
                    Fv = self._riemann(own["q"], own["f"], tr[opp[f]]["q"][o:o + 1], tr[opp[f]]["f"][o:o + 1],
                                       z, own_minus, nrm[f], hn)
                elif nb[0] == "coarse":
                    o, sp = nb[1], nb[2]
                    oidx = [kk for kk, c in enumerate(self.leaves) if c[0] == lv - 1].index(o)
                    sub = self._lts_sub[lv - 1][kstep]
                    cq = self._prolong_face(sub[opp[f]]["q"][oidx:oidx + 1], sp)
                    cf = self._prolong_face(sub[opp[f]]["f"][oidx:oidx + 1], sp)
                    Fv = self._riemann(own["q"], own["f"], cq, cf, z, own_minus, nrm[f], hn)
                    acc = self._lts_acc[(o, opp[f])]
                    acc[sp] = acc[sp] + Fv / 3.0
                else:  # three finer neighbours: their three sub-step fluxes, averaged, restricted
                    Fv = self._restrict_face(self._lts_acc[(k, f)])
                Fst[f][a] = Fv[0]
        w, p0, p1 = b.w, b.phi0, b.phi1
        Vx = (w[:, None] * b.D) / w[None, :]
        hx, hy = self.h(lv)
        vol = (torch.einsum("pi,cvjp->cvji", Vx, tavg["Fbar"]) / hx
               + torch.einsum("pj,cvpi->cvji", Vx, tavg["Gbar"]) / hy)
        FE, FW, GN, GS = Fst["E"], Fst["W"], Fst["N"], Fst["S"]
        face = ((p1[None, None, None, :] * FE[:, :, :, None] - p0[None, None, None, :] * FW[:, :, :, None])
                / (hx * w[None, None, None, :])
                + (p1[None, None, :, None] * GN[:, :, None, :] - p0[None, None, :, None] * GS[:, :, None, :])
                / (hy * w[None, None, :, None]))
        self._lts_u[idx] = self._lts_u[idx] + dtl * (vol - face + tavg["Sbar"])

    def _face_z(self, leaf, f):
        lv, ix, iy = leaf
        hx, hy = self.h(lv)
        if f in "EW":
            return (self.y0 + (iy + self.b.xi) * hy)[None, :]
        return torch.full((1, self.b.n), self.y0 + (iy + (1 if f == "N" else 0)) * hy, dtype=DTYPE)

    def _riemann(self, q_own, f_own, q_oth, f_oth, z, own_minus, nrm, h):
        if own_minus:
            return self.ref.riemann(q_own, f_own, q_oth, f_oth, z, z, nrm, h)
        return self.ref.riemann(q_oth, f_oth, q_own, f_own, z, z, nrm, h)

    def _prolong_face(self, a, s):
        """Face data a[1, v, q] of a coarse face evaluated on its third s."""
        return torch.einsum("mq,cvq->cvm", self.Pro[s], a)

    def _restrict_face(self, subs):
        """L2 restriction of three fine face fluxes onto the coarse face basis."""
        w = self.b.w
        acc = 0.0
        for s, F in enumerate(subs):
            # int_coarse phi_q F = sum_s (1/3) sum_m w_m phi_q((s + xi_m)/3) F_s[m]
            acc = acc + torch.einsum("mq,m,cvm->cvq", self.Pro[s], w, F) / 3.0
        return acc / w[None, None, :]

    # -------------------------------------------------------------- transfer
    def prolong_cell(self, u):
        """Children (a, b) = (x, y position) of parent nodal data u[v, j, i]."""
        return {(a, bb): torch.einsum("jr,iq,vrq->vji", self.Pro[bb], self.Pro[a], u)
                for a in range(3) for bb in range(3)}

    def restrict_cell(self, kids):
        """Parent nodal values: L2 projection of the 9 children (GL on each)."""
        w = self.b.w
        acc = 0.0
        for (a, bb), uc in kids.items():
            acc = acc + torch.einsum("lj,mi,l,m,vlm->vji", self.Pro[bb], self.Pro[a], w, w, uc) / 9.0
        return acc / (w[:, None] * w[None, :])[None]

    # -------------------------------------------------------------- adaptation
    def _balanced_refine(self, refine):
        refine = set(refine)
        changed = True
        while changed:
            changed = False
            for k in list(refine):
                lv, ix, iy = self.leaves[k]
                for f in "EWNS":
                    nb = self.neighbour(self.leaves[k], f)
                    if nb[0] == "coarse" and nb[1] not in refine:
                        refine.add(nb[1])
                        changed = True
        return refine

    def adapt(self, u, flags):
        """Apply refine (+1) / coarsen (-1) flags per leaf; returns the new state."""
        flags = [int(x) for x in flags]
        refine = {k for k, fl in enumerate(flags) if fl > 0 and self.leaves[k][0] < self.max_level}
        refine = self._balanced_refine(refine)
        # sibling groups all flagged -1 (and none refined)
        groups = {}
        for k, (lv, ix, iy) in enumerate(self.leaves):
            if lv > 0:
                groups.setdefault((lv - 1, ix // 3, iy // 3), []).append(k)
        new_levels = {}
        for k, c in enumerate(self.leaves):
            new_levels[k] = c[0] + (1 if k in refine else 0)
        coarsen = []
        for parent, ks in groups.items():
            if len(ks) != 9 or any(flags[k] >= 0 or k in refine for k in ks):
                continue
            # A3: after coarsening, the parent may not touch a leaf two levels finer
            ok = True
            plv, pix, piy = parent
            for k in ks:
                for f in "EWNS":
                    nb = self.neighbour(self.leaves[k], f)
                    if nb[0] == "fine":
                        ok = False
                    elif nb[0] == "conf" and nb[1] not in ks and new_levels[nb[1]] > plv + 1:
                        ok = False
            if ok:
                coarsen.append((parent, ks))
        coarse_members = {k for _, ks in coarsen for k in ks}
        new = {}
        for k, c in enumerate(self.leaves):
            if k in coarse_members:
                continue
            if k in refine:
                lv, ix, iy = c
                kids = self.prolong_cell(u[k])
                for (a, bb), uc in kids.items():
                    new[(lv + 1, 3 * ix + a, 3 * iy + bb)] = uc
            else:
                new[c] = u[k]
        for parent, ks in coarsen:
            kids = {}
            for k in ks:
                lv, ix, iy = self.leaves[k]
                kids[(ix % 3, iy % 3)] = u[k]
            new[parent] = self.restrict_cell(kids)
        self.leaves = list(new.keys())
        self._index()
        return torch.stack([new[c] for c in self.leaves])

    def integral(self, u):
        w = self.b.w
        tot = 0.0
        for lv, idx, view in self.level_views():
            hx, hy = self.h(lv)
            tot = tot + torch.einsum("j,i,cvji->v", w, w, u[idx]) * hx * hy
        return tot

    def interpolate_field(self, fn):
        """Nodal values of an analytic field fn(X, Y) -> [c, 4, n, n]."""
        X, Y = self.node_coords()
        return torch.stack(fn(X, Y), 1)
