"""Unrolled message passing in PyTorch FP64, for reference gradients.

TEST INFRASTRUCTURE ONLY -- imported by tests, never by the product library.

Section 4.4 writes K iterations as a composition s^K = h^K o ... o h^1 (s^0)
of almost-everywhere differentiable steps, so the system cost f(p^K) after K
iterations can be differentiated with respect to the problem data; Section
5.5 differentiates it with respect to generator capacities.  This module
repeats the iteration of Section 3.2 (the same steps as ``oracle.mp``) with
PyTorch tensors so that autograd gives the reference gradient of

    f(p^K) = sum_gen (a p^2 + b p) + sum_curtailable voll (p + P)

    + sum_batteries cost . delta

with respect to load power P [D][T], generator capacity pmax [G][T] and line
limits u [L], for fixed penalties (no adaptation: the adaptive rule is a
discrete decision).  Ramp-limited generators and batteries take their prox
from the Appendix D inner ADMM exactly as ``oracle.mp`` runs it (the same
constraint rows, ``omega = rho'``, ``(beta, lambda)`` carried across outer
iterations from zero); autograd then differentiates through the inner
iterations, and a ramp generator's capacity enters through the right-hand
side of its ``p_t <= pmax_t`` rows; ``delta`` is the discharge of the last
inner iterate.  Clipping follows torch.clamp: the value passes its gradient
where lo <= x <= hi, a bound receives it where x leaves the interval on its
side; the inner projection ``min(alpha + lambda, 0)`` is a clamp with upper
bound 0.
"""
from __future__ import annotations

import numpy as np
import torch

from .mp import Network, inner_matrix, ramp_rows, storage_layout, storage_rows


class Unrolled:
    """The iteration of Section 3.2 as a differentiable function of (P, pmax, u)."""

    def __init__(self, case, rho_p=1.0, rho_theta=1.0):
        net = Network(case)
        self.net = net
        self.case = case
        self.rho_p, self.rho_th = float(rho_p), float(rho_theta)
        t = lambda a, dt=torch.float64: torch.as_tensor(np.asarray(a), dtype=dt)
        self.tn = t(net.term_node, torch.long)
        self.tn_ph = self.tn[:2 * net.L]
        cnt = np.asarray(net.count, float)
        cth = np.asarray(net.count_th, float)
        self.cnt = t(cnt)
        self.cnt_th = t(np.where(cth > 0, cth, 1.0))
        self.has_th = t(cth > 0, torch.bool)
        self.active = t(net.active)
        self.line_b = t(net.line_b)
        self.gen_a, self.gen_b = t(net.gen_a), t(net.gen_b)
        self.gen_pmin = t(net.gen_pmin)
        self.load_voll = t(net.load_voll)
        self.is_fixed = t(net.is_fixed, torch.bool)
        self.hvdc_u = t(net.hvdc_u)
        # inner-ADMM devices (Appendix D), factored once: the penalties are fixed
        T = net.T
        rho_d = net.Kp * self.rho_p
        self.ramp_idx = np.nonzero(net.is_ramp)[0]
        if len(self.ramp_idx):
            A, _, eq = ramp_rows(np.zeros(T), np.zeros(T), 0.0)
            Qd = np.repeat(net.gen_a[self.ramp_idx][:, None], T, axis=1)
            self.ramp_A, self.ramp_eq = t(A), t(eq, torch.bool)
            self.ramp_Minv = t(np.linalg.inv(inner_matrix(Qd, rho_d, rho_d, A, T)))
            # right-hand sides without the pmax rows, which come from the parameter
            self.ramp_h_rest = t(np.stack([ramp_rows(net.gen_pmin[g], net.gen_pmax[g], net.gen_ramp[g])[1][T:]
                                           for g in self.ramp_idx]))
            self.ramp_q = t(np.repeat(net.gen_b[self.ramp_idx][:, None], T, axis=1))
        self.stor = []
        if net.B:
            groups = {}
            for b in range(net.B):
                groups.setdefault(float(net.stor_eff[b]), []).append(b)
            _, _, sdl, _ = storage_layout(T)
            self.stor_sdl = sdl
            for eff, members in groups.items():
                mb = np.asarray(members)
                A, _, eq = storage_rows(T, eff, 0.0, 0.0)
                h = np.stack([storage_rows(T, eff, net.stor_P[b], net.stor_dur[b])[1] for b in mb])
                q = np.zeros((len(mb), 4 * T + 1))
                q[:, sdl] = net.stor_cost[mb][:, None]
                Minv = np.linalg.inv(inner_matrix(np.zeros((len(mb), 4 * T + 1)), rho_d, rho_d, A, T))
                self.stor.append(dict(members=t(mb, torch.long), A=t(A), eq=t(eq, torch.bool), h=t(h),
                                      q=t(q), Minv=t(Minv), cost=t(net.stor_cost[mb])))

    @staticmethod
    def _inner(x, A, h, eq, q, rho, Minv, beta, lam, n_iter):
        """The inner ADMM of ``oracle.mp.inner_admm`` (Appendix D, omega =
        rho) on tensors, so that autograd differentiates through it."""
        n_p = x.shape[1]
        z = None
        for _ in range(n_iter):
            rhs = -q + rho * ((h + beta - lam) @ A)
            rhs = torch.cat([rhs[:, :n_p] + rho * x, rhs[:, n_p:]], dim=1)
            z = torch.einsum("dij,dj->di", Minv, rhs)
            alpha = z @ A.T - h
            s = alpha + lam
            beta = torch.where(eq[None, :], torch.zeros_like(s), torch.clamp(s, max=0.0))
            lam = lam + alpha - beta
        return z, beta, lam

    def params(self, requires_grad=True):
        """The data the cost is differentiated with respect to (loads,
        generator capacities, line limits: the sensitivities of Section 5.5),
        as leaf tensors."""
        n = self.net
        out = dict(load_p=torch.tensor(n.load_p, dtype=torch.float64),
                   gen_pmax=torch.tensor(n.gen_pmax, dtype=torch.float64),
                   line_u=torch.tensor(n.line_u, dtype=torch.float64))
        for v in out.values():
            v.requires_grad_(requires_grad)
        return out

    def _node_mean(self, z, phase):
        """Node averages (Eq. average-op) of terminal values z [Kp, J or 2L, T]."""
        n = self.net
        idx = self.tn_ph if phase else self.tn
        s = torch.zeros((z.shape[0], n.N, z.shape[2]), dtype=z.dtype).index_add(1, idx, z)
        if phase:
            return torch.where(self.has_th[None, :, None], s / self.cnt_th[None, :, None], torch.zeros_like(s))
        return s / self.cnt[None, :, None]

    def run(self, prm, K, inner_iters=10):
        """Iterate K times from zero at fixed penalties (the unrolled map of
        Section 4.4, each step the message-passing iteration of Section 3.2);
        returns (cost f(p^K), final p_dev [S][T])."""
        n = self.net
        Kp, J, L, T = n.Kp, n.J, n.L, n.T
        G, D = n.G, n.D
        rp, rt = self.rho_p, self.rho_th
        rho_d = Kp * rp
        p = torch.zeros((Kp, J, T), dtype=torch.float64)
        th = torch.zeros((Kp, 2 * L, T), dtype=torch.float64)
        v = torch.zeros_like(th)
        u = torch.zeros((Kp, n.N, T), dtype=torch.float64)
        act = self.active[:, :, None].to(torch.bool)
        ulim = prm["line_u"][None, :, None] * self.active[:, :, None]
        bs = torch.where(act, self.line_b[None, :, None], torch.ones_like(self.line_b[None, :, None]))
        sd = slice(2 * L, J)
        f64 = torch.float64
        if len(self.ramp_idx):
            ri = torch.as_tensor(self.ramp_idx, dtype=torch.long)
            m = self.ramp_A.shape[0]
            r_beta = torch.zeros((len(ri), m), dtype=f64)
            r_lam = torch.zeros((len(ri), m), dtype=f64)
            r_h = torch.cat([prm["gen_pmax"][ri], self.ramp_h_rest], dim=1)
        s_state = [(torch.zeros((len(g["members"]), g["A"].shape[0]), dtype=f64),
                    torch.zeros((len(g["members"]), g["A"].shape[0]), dtype=f64)) for g in self.stor]
        s_z = [None] * len(self.stor)
        for _ in range(K):
            pbar_n = self._node_mean(p, False)
            thbar_n = self._node_mean(th, True)
            pbar = pbar_n[:, self.tn, :]
            thbar = thbar_n[:, self.tn_ph, :]
            uj = u[:, self.tn, :]
            x = p - pbar - uj
            y = thbar - v
            # step 1: line prox (Section 4.2), outaged lines decouple
            x1, x2, y1, y2 = x[:, :L], x[:, L:2 * L], y[:, :L], y[:, L:]
            num = rp * (x2 - x1) + rt * (y1 - y2) / (2 * bs)
            den = 2 * rp + rt / (2 * bs * bs)
            p2 = torch.clamp(num / den, min=-ulim, max=ulim)
            mid = 0.5 * (y1 + y2)
            th1 = torch.where(act, mid + p2 / (2 * bs), y1)
            th2 = torch.where(act, mid - p2 / (2 * bs), y2)
            p2 = torch.where(act, p2, torch.zeros_like(p2))
            # step 2: devices shared by all contingencies, weight (K+1) rho_p
            X = p[0, sd] - (pbar[:, sd] + uj[:, sd]).mean(dim=0)
            Xg, Xl = X[:G], X[G:G + D]
            pg = torch.clamp((rho_d * Xg - self.gen_b[:, None]) / (2 * self.gen_a[:, None] + rho_d),
                             min=self.gen_pmin, max=prm["gen_pmax"])
            pl = torch.clamp((rho_d * Xl - self.load_voll[:, None]) / rho_d, min=-prm["load_p"],
                             max=torch.zeros_like(Xl))
            pl = torch.where(self.is_fixed[:, None], -prm["load_p"], pl)
            if len(self.ramp_idx):
                z, r_beta, r_lam = self._inner(Xg[ri], self.ramp_A, r_h, self.ramp_eq, self.ramp_q, rho_d,
                                               self.ramp_Minv, r_beta, r_lam, inner_iters)
                pg = pg.index_put((ri,), z[:, :T])
            parts = [pg, pl]
            if self.stor:
                Xb = X[G + D:G + D + n.B]
                pb = torch.zeros_like(Xb)
                for i, g in enumerate(self.stor):
                    z, bt, lm = self._inner(Xb[g["members"]], g["A"], g["h"], g["eq"], g["q"], rho_d, g["Minv"],
                                            s_state[i][0], s_state[i][1], inner_iters)
                    s_state[i] = (bt, lm)
                    s_z[i] = z
                    pb = pb.index_put((g["members"],), z[:, :T])
                parts.append(pb)
            if n.H:
                # HVDC links: p2 = clip((x2 - x1) / 2, -u, u), p1 = -p2 (oracle.mp.prox_hvdc)
                h0 = G + D + n.B
                xh = X[h0:h0 + 2 * n.H].reshape(n.H, 2, T)
                hu = self.hvdc_u[:, None]
                p2h = torch.clamp((xh[:, 1] - xh[:, 0]) / 2, min=-hu, max=hu)
                parts.append(torch.stack([-p2h, p2h], dim=1).reshape(2 * n.H, T))
            pd = torch.cat(parts, dim=0)
            p = torch.cat([-p2, p2, pd[None].expand(Kp, -1, -1)], dim=1)
            th = torch.cat([th1, th2], dim=1)
            # step 3: scaled price updates
            pbar_new = self._node_mean(p, False)
            thbar_new = self._node_mean(th, True)
            u = u + pbar_new
            v = v + th - thbar_new[:, self.tn_ph, :]
        pd = p[0, sd]
        pg, pl = pd[:G], pd[G:G + D]
        f = (self.gen_a[:, None] * pg * pg + self.gen_b[:, None] * pg).sum()
        cur = ~self.is_fixed
        f = f + (self.load_voll[cur, None] * (pl[cur] + prm["load_p"][cur])).sum()
        for g, z in zip(self.stor, s_z):
            if z is not None:
                f = f + (g["cost"][:, None] * z[:, self.stor_sdl]).sum()
        return f, pd
