"""Unrolled message passing in PyTorch FP64, for reference gradients.

TEST INFRASTRUCTURE ONLY -- imported by tests, never by the product library.

Section 4.4 writes K iterations as a composition s^K = h^K o ... o h^1 (s^0)
of almost-everywhere differentiable steps, so the system cost f(p^K) after K
iterations can be differentiated with respect to the problem data; Section
5.5 differentiates it with respect to generator capacities.  This module
repeats the iteration of Section 3.2 (the same steps as ``oracle.mp``) with
PyTorch tensors so that autograd gives the reference gradient of

    f(p^K) = sum_gen (a p^2 + b p) + sum_curtailable voll (p + P)

with respect to load power P [D][T], generator capacity pmax [G][T] and line
limits u [L], for fixed penalties (no adaptation: the adaptive rule is a
discrete decision).  Scope: devices with a closed-form prox (generators
without ramp limits, fixed and curtailable loads); ramp-limited generators
and batteries are not covered.  Clipping follows torch.clamp: the value
passes its gradient where lo <= x <= hi, a bound receives it where x leaves
the interval on its side.
"""
from __future__ import annotations

import numpy as np
import torch

from .mp import Network


class Unrolled:
    """The iteration of Section 3.2 as a differentiable function of (P, pmax, u)."""

    def __init__(self, case, rho_p=1.0, rho_theta=1.0):
        net = Network(case)
        if net.B or np.any(net.is_ramp):
            raise ValueError("the unrolled reference covers closed-form devices only "
                             "(no batteries, no ramp limits)")
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

    def params(self, requires_grad=True):
        """The data the cost is differentiated with respect to, as leaf tensors."""
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

    def run(self, prm, K):
        """Iterate K times from zero; returns (cost f(p^K), final p_dev [S][T])."""
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
            pd = torch.cat([pg, pl], dim=0)
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
        return f, pd
