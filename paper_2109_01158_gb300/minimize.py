"""L-BFGS minimisation of J(v) driven by the energy + gradient kernels.

The paper minimises with MATLAB's trust-region method (Sec. 7); this module replaces it by
limited-memory BFGS (Nocedal & Wright, Numerical Optimization, Alg. 7.4 two-loop recursion)
with a bracketing line search.  A step is accepted when it satisfies the weak Wolfe
conditions or -- once energy differences reach the rounding level of J -- the approximate
Wolfe conditions of Hager & Zhang (SIAM J. Optim. 16, 2005): J does not rise above
J + eps_f |J| and the directional derivative satisfies sigma g.d <= g_new.d <= (2 c1 - 1) g.d.
Iterates stay on the device; Dirichlet dofs never move because the gradient is 0 there.  A
trial point with det F <= 0 has J = +Inf and is rejected like any point without decrease.

`lbfgs` runs one minimisation through an evaluator `ev(v) -> (J, g)`; `lbfgs_batched` runs
many instances in lockstep, evaluating every active instance's trial point in one batched
launch (fe_batch_energy_gradient) per line-search round.  `newton_cg` is a trust-region
Newton-CG method on the kernels' Hessian-vector products (fe_hessian_vector), with the inner
CG on the host (torch) or on the device (fe_cg_steihaug); `nested_newton` runs it on a
sequence of uniformly refined meshes, each started from the previous minimiser.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch


@dataclass
class LBFGSResult:
    v: torch.Tensor
    J: float
    gnorm: float
    iters: int
    evals: int
    converged: bool
    seconds: float
    history: list = field(default_factory=list)   # (J, ||g||_inf) per iteration
    checkpoint: dict | None = None                # LbfgsJob.checkpoint() at the stop, when asked for


def _gnorm(g):
    return float(g.abs().max().item()) if g.numel() else 0.0


class _LineSearch:
    """Bracketing search for a step t > 0 along a descent direction d (phi(t) = J(v + t d)).

    Accepts t when phi satisfies the weak Wolfe conditions -- sufficient decrease
    phi(t) <= phi(0) + c1 t phi'(0) and curvature phi'(t) >= sigma phi'(0) -- or, once energy
    differences are at the rounding level of J, the approximate Wolfe conditions of Hager &
    Zhang: phi(t) <= phi(0) + eps_f |phi(0)| and sigma phi'(0) <= phi'(t) <= (2 c1 - 1) phi'(0).
    A step that fails the decrease test (or gives J = +Inf) becomes the upper end of the
    bracket; a step that passes it but is too short becomes the lower end.  Without an upper
    end the step doubles; inside a bracket the next step is the secant root of phi' when both
    ends carry derivatives of opposite sign (kept at least 10% of the bracket from each end),
    else the midpoint."""

    def __init__(self, J, gd, c1, sigma, eps_f, t0=1.0):
        self.J, self.gd = J, gd
        self.c1, self.sigma, self.eps_f = c1, sigma, eps_f
        self.lo, self.d_lo = 0.0, gd
        self.hi, self.d_hi = math.inf, None
        self.t = t0

    def update(self, J_new, gd_new):
        """Feed phi(t), phi'(t) of the current trial; True when t is accepted."""
        t = self.t
        if not (math.isfinite(J_new) and math.isfinite(gd_new)):
            self.hi, self.d_hi = t, None
        else:
            armijo = J_new <= self.J + self.c1 * t * self.gd
            approx = (J_new <= self.J + self.eps_f * abs(self.J)
                      and gd_new <= (2.0 * self.c1 - 1.0) * self.gd)
            if not (armijo or approx):
                self.hi, self.d_hi = t, gd_new
            elif gd_new >= self.sigma * self.gd:
                return True
            else:
                self.lo, self.d_lo = t, gd_new
        if math.isinf(self.hi):
            self.t = 2.0 * t
            return False
        lo, hi, w = self.lo, self.hi, self.hi - self.lo
        nt = 0.5 * (lo + hi)
        if self.d_hi is not None and self.d_lo < 0.0 < self.d_hi:
            nt = lo - self.d_lo * w / (self.d_hi - self.d_lo)
            nt = min(max(nt, lo + 0.1 * w), hi - 0.1 * w)
        self.t = nt
        return False


class _State:
    """L-BFGS state of one instance (m most recent pairs on the device)."""

    def __init__(self, v, J, g, m):
        self.v, self.J, self.g = v, J, g
        self.S, self.Y, self.R = [], [], []
        self.m = m
        self.iters = 0
        self.evals = 1
        self.done = False
        self.history = []

    def direction(self):
        """Two-loop recursion; the initial Hessian scaling is s.y / y.y of the newest pair, and
        the very first step has unit length.  Falls back to -g (memory cleared) when the
        result is not a descent direction."""
        q = -self.g
        alphas = []
        for s, y, rho in zip(reversed(self.S), reversed(self.Y), reversed(self.R)):
            a = rho * torch.dot(s, q)
            alphas.append(a)
            q = q - a * y
        if self.S:
            s, y = self.S[-1], self.Y[-1]
            q = q * (torch.dot(s, y) / torch.dot(y, y))
        else:
            gn = torch.linalg.vector_norm(self.g)
            q = q / torch.clamp(gn, min=1e-300)
        for (s, y, rho), a in zip(zip(self.S, self.Y, self.R), reversed(alphas)):
            b = rho * torch.dot(y, q)
            q = q + s * (a - b)
        gd = float(torch.dot(self.g, q).item())
        if not gd < 0.0 and self.S:
            self.S.clear(), self.Y.clear(), self.R.clear()
            return self.direction()
        return q, gd

    def accept(self, v_new, J_new, g_new):
        s = v_new - self.v
        y = g_new - self.g
        sy = float(torch.dot(s, y).item())
        if sy > 0.0:          # weak Wolfe guarantees s.y > 0 unless the step is rounding-level
            self.S.append(s)
            self.Y.append(y)
            self.R.append(1.0 / sy)
            if len(self.S) > self.m:
                self.S.pop(0), self.Y.pop(0), self.R.pop(0)
        self.v, self.J, self.g = v_new, J_new, g_new
        self.iters += 1


class _DeviceState(_State):
    """_State with the pairs and the direction on the device (fem.LbfgsMemory: the compact
    representation of the same inverse Hessian, in fused kernels)."""

    def __init__(self, v, J, g, m):
        super().__init__(v, J, g, m)
        from .fem import LbfgsMemory
        self.mem = LbfgsMemory(v.numel(), m, v.device)

    def direction(self):
        d, gd = self.mem.direction(self.g)
        if not gd < 0.0 and self.mem.pairs() > 0:
            self.mem.reset()
            d, gd = self.mem.direction(self.g)
        return d, gd

    def accept(self, v_new, J_new, g_new):
        self.mem.update(v_new, self.v, g_new, self.g)
        self.v, self.J, self.g = v_new, J_new, g_new
        self.iters += 1

    def accept_step(self, v_new, J_new, g_new):
        """accept(), the next direction() and ||g_new||_inf in one host round trip: returns
        (d, g_new.d, ||g_new||_inf)."""
        d, _, gd, gmax = self.mem.step(v_new, self.v, g_new, self.g)
        self.v, self.J, self.g = v_new, J_new, g_new
        self.iters += 1
        if not gd < 0.0 and self.mem.pairs() > 0:
            self.mem.reset()
            d, gd = self.mem.direction(self.g)
        return d, gd, gmax

    def close(self):
        self.mem.close()


def _noise(ev, eps_f):
    """Relative rounding level of J: the caller's, else the evaluator's `eps_f`, else 1e-10."""
    return eps_f if eps_f is not None else getattr(ev, "eps_f", 1e-10)


class LbfgsJob:
    """One L-BFGS minimisation as a state machine, so that a loop can drive many at once:
    trial() is the point whose (J, g) the job needs next, feed(J, g) consumes them.  The first
    trial is v0; then each iteration computes a direction and feeds line-search trials until
    one is accepted.  done turns True when ||g||_inf <= tol, the iteration limit is reached, a
    direction is not a descent direction, or a line search gives up after max_evals_per_iter
    trials; result() then returns the LBFGSResult.  Driving one job with ev gives `lbfgs`."""

    def __init__(self, v0, *, m: int = 10, gtol: float = 1e-6, relative: bool = False, max_iter: int = 20000,
                 c1: float = 1e-4, sigma: float = 0.9, eps_f: float = 1e-10, max_evals_per_iter: int = 60,
                 device_memory: bool = False, resume: dict | None = None, keep_checkpoint: bool = False):
        self.v0 = v0
        self.device_memory = device_memory and v0.is_cuda
        self.m, self.gtol, self.relative, self.max_iter = m, gtol, relative, max_iter
        self.c1, self.sigma, self.eps_f, self.max_evals = c1, sigma, eps_f, max_evals_per_iter
        self.keep_checkpoint = keep_checkpoint
        self.final_checkpoint = None
        self.st = None
        self.done = False
        self.t0 = time.perf_counter()
        self.seconds = 0.0
        self._trial = v0
        if resume is not None:
            self._resume(resume)

    # ---- checkpoint / resume (device memory only) ---------------------------------------
    def checkpoint(self) -> dict:
        """The state between two iterations, on the host: iterate, J, g, the L-BFGS pairs and
        their products, counters and history.  A job built with resume=<this> continues with
        bitwise the iterates this one would have produced.  Only between iterations (after
        construction from a resume, or when the job stopped at max_iter with keep_checkpoint)."""
        if not self.device_memory:
            raise ValueError("checkpoints need the device L-BFGS memory (device_memory=True)")
        st = self.st
        if st is None:
            raise ValueError("no iteration yet")
        return {"v": st.v.detach().cpu().numpy().copy(), "J": float(st.J), "g": st.g.detach().cpu().numpy().copy(),
                "gn": float(self.gn), "tol": float(self.tol), "iters": int(st.iters), "evals": int(st.evals),
                "history": list(st.history), "m": int(self.m), "memory": st.mem.save()}

    def _resume(self, ck: dict):
        if not self.device_memory:
            raise ValueError("resuming needs the device L-BFGS memory (device_memory=True, a CUDA v0)")
        if int(ck["m"]) != self.m or ck["v"].shape != tuple(self.v0.shape):
            raise ValueError("checkpoint does not match this problem (m or size)")
        dev = self.v0.device
        v = torch.from_numpy(ck["v"]).to(dev)
        g = torch.from_numpy(ck["g"]).to(dev)
        self.st = _DeviceState(v, float(ck["J"]), g, self.m)
        self.st.mem.restore(ck["memory"])
        self.st.iters, self.st.evals = int(ck["iters"]), int(ck["evals"])
        self.st.history = list(ck["history"])
        self.gn, self.tol = float(ck["gn"]), float(ck["tol"])
        self._next_iteration()


    def trial(self):
        return self._trial

    def search_direction(self):
        """The direction of the current line search (None before the first evaluation)."""
        return None if (self.st is None or self.done) else self.d

    def feed(self, J, g, gd=None):
        """J (a float or a device scalar) and g at trial(); gd: g.d along search_direction()
        when the caller has it already (else it is computed here, read together with J)."""
        if self.st is not None and gd is None:
            gdt = torch.dot(g, self.d)
            if isinstance(J, torch.Tensor):
                J, gd = torch.stack([J.reshape(()).to(gdt.dtype), gdt]).tolist()
            else:
                gd = float(gdt.item())
        J = float(J)
        if self.st is None:
            self.st = (_DeviceState if self.device_memory else _State)(self.v0.clone(), J, g, self.m)
            self.gn = _gnorm(g)
            self.tol = self.gtol * (self.gn if self.relative else 1.0)
            self.st.history.append((J, self.gn))
            self._next_iteration()
            return
        st = self.st
        st.evals += 1
        if self.ls.update(J, float(gd)):
            if isinstance(st, _DeviceState):
                d, gdn, self.gn = st.accept_step(self._trial, J, g)
                st.history.append((st.J, self.gn))
                self._next_iteration((d, gdn))
            else:
                st.accept(self._trial, J, g)
                self.gn = _gnorm(st.g)
                st.history.append((st.J, self.gn))
                self._next_iteration()
            return
        self.n_search += 1
        if self.n_search >= self.max_evals:
            self._finish()
        else:
            self._trial = st.v + self.ls.t * self.d

    def _next_iteration(self, direction=None):
        st = self.st
        if not (self.gn > self.tol and st.iters < self.max_iter):
            self._finish()
            return
        self.d, gd = direction if direction is not None else st.direction()
        if not gd < 0.0:
            self._finish()
            return
        self.ls = _LineSearch(st.J, gd, self.c1, self.sigma, self.eps_f)
        self.n_search = 0
        self._trial = st.v + self.ls.t * self.d

    def _finish(self):
        self.done = True
        self._trial = None
        self.seconds = time.perf_counter() - self.t0
        if isinstance(self.st, _DeviceState):
            if self.keep_checkpoint:
                self.final_checkpoint = self.checkpoint()
            self.st.close()

    def result(self) -> LBFGSResult:
        st = self.st
        return LBFGSResult(st.v, st.J, self.gn, st.iters, st.evals, self.gn <= self.tol, self.seconds, st.history,
                           self.final_checkpoint)


def lbfgs(ev, v0: torch.Tensor, *, m: int = 10, gtol: float = 1e-6, relative: bool = False,
          max_iter: int = 20000, c1: float = 1e-4, sigma: float = 0.9, eps_f: float | None = None,
          max_evals_per_iter: int = 60, device_memory: bool = False, resume: dict | None = None,
          checkpoint: bool = False) -> LBFGSResult:
    """Minimise J from v0.  Stops when ||g||_inf <= gtol (times ||g0||_inf if relative), or when
    a line search finds no acceptable step (converged is then False).  eps_f is the relative
    rounding level of the evaluated J used by the approximate Wolfe test.  device_memory keeps
    the pairs and computes the directions in the library's kernels (fe_lbfgs; CUDA v0 only)
    instead of torch vector operations.  checkpoint=True returns the state at the stop in
    result.checkpoint (device memory only); resume=<such a state> continues from it (v0 then
    only gives the device and size), with bitwise the iterates of an uninterrupted run, and
    max_iter counts the iterations of the whole run."""
    job = LbfgsJob(v0, m=m, gtol=gtol, relative=relative, max_iter=max_iter, c1=c1, sigma=sigma,
                   eps_f=_noise(ev, eps_f), max_evals_per_iter=max_evals_per_iter, device_memory=device_memory,
                   resume=resume, keep_checkpoint=checkpoint)
    while not job.done:
        J, g = ev(job.trial())
        job.feed(J, g)
    return job.result()


def lbfgs_batched(batch_eval, v0s, *, m: int = 10, gtol: float = 1e-6, relative: bool = False,
                  max_iter: int = 20000, c1: float = 1e-4, sigma: float = 0.9, eps_f: float | None = None,
                  max_evals_per_iter: int = 60, device_memory: bool = False):
    """Several L-BFGS instances driven together.  batch_eval(list of (k, v)) -> list of (J, g)
    evaluates the pending trial point of every unfinished instance in one batched launch; each
    instance follows exactly the iterates `lbfgs` would produce for it alone."""
    eps_f = _noise(batch_eval, eps_f)
    jobs = [LbfgsJob(v, m=m, gtol=gtol, relative=relative, max_iter=max_iter, c1=c1, sigma=sigma, eps_f=eps_f,
                     max_evals_per_iter=max_evals_per_iter, device_memory=device_memory) for v in v0s]
    while True:
        active = [k for k, j in enumerate(jobs) if not j.done]
        if not active:
            break
        res = batch_eval([(k, jobs[k].trial()) for k in active])
        for k, (J, g) in zip(active, res):
            jobs[k].feed(J, g)
    return [j.result() for j in jobs]


@dataclass
class NewtonResult:
    v: torch.Tensor
    J: float
    gnorm: float
    iters: int
    evals: int
    hvps: int
    converged: bool
    seconds: float
    history: list = field(default_factory=list)   # (J, ||g||_inf, CG iterations) per iteration


def _to_boundary(z, d, radius):
    """tau >= 0 with ||z + tau d|| = radius."""
    dd = float(torch.dot(d, d).item())
    zd = float(torch.dot(z, d).item())
    zz = float(torch.dot(z, z).item())
    disc = max(zd * zd + dd * (radius * radius - zz), 0.0)
    return (-zd + math.sqrt(disc)) / max(dd, 1e-300)


def _cg_steihaug(g, hv, radius, tol, max_cg, history=None):
    """Steihaug's truncated CG (Nocedal & Wright, Alg. 7.2) for min g.z + z.Hz/2 within
    ||z|| <= radius.  Returns (z, Hz, iterations, hit_boundary); `history`, when a list, gets
    the residual norm after every step."""
    z = torch.zeros_like(g)
    Hz = torch.zeros_like(g)
    r = g.clone()
    d = -r
    rr = float(torch.dot(r, r).item())
    if math.sqrt(rr) <= tol:
        return z, Hz, 0, False
    for k in range(1, max_cg + 1):
        Hd = hv(d)
        dHd = float(torch.dot(d, Hd).item())
        if not dHd > 0.0:
            tau = _to_boundary(z, d, radius)
            return z + tau * d, Hz + tau * Hd, k, True
        alpha = rr / dHd
        z_new = z + alpha * d
        if float(torch.linalg.vector_norm(z_new).item()) >= radius:
            tau = _to_boundary(z, d, radius)
            return z + tau * d, Hz + tau * Hd, k, True
        z, Hz = z_new, Hz + alpha * Hd
        r = r + alpha * Hd
        rr_new = float(torch.dot(r, r).item())
        if history is not None:
            history.append(math.sqrt(rr_new))
        if math.sqrt(rr_new) <= tol:
            return z, Hz, k, False
        d = -r + (rr_new / rr) * d
        rr = rr_new
    return z, Hz, max_cg, False


def newton_cg(ev, hvp, v0: torch.Tensor, *, gtol: float = 1e-6, relative: bool = False,
              max_iter: int = 1000, max_cg: int = 5000, eta_max: float = 0.1,
              eps_f: float | None = None, radius_max: float = 1e30, cg=None) -> NewtonResult:
    """Trust-region Newton-CG (Nocedal & Wright, Alg. 4.1 with Steihaug's CG), the analogue
    of the trust-region method the paper minimises with (Sec. 7), driven by the kernels'
    Hessian-vector products hvp(v, w) -> Hw.  The inner CG stops at ||r|| <= eta ||g||,
    eta = min(eta_max, sqrt(||g|| / ||g_0||)), at the trust-region boundary, or at a direction
    of non-positive curvature (the p-Laplacian's Hessian vanishes where grad v = 0).  The
    first radius is the length of the Cauchy step.  A step is accepted when the ratio of
    actual to predicted decrease exceeds 1e-4, or -- at the rounding level of J -- when J
    does not rise above it and ||g|| decreases.  cg(v, g, radius, tol, max_cg) -> (z, Hz, k,
    hit_boundary) replaces the Python CG over hvp (e.g. the device solver of mesh_cg)."""
    t0 = time.perf_counter()
    eps_f = _noise(ev, eps_f)
    J, g = ev(v0)
    J = float(J)
    v = v0.clone()
    gn = _gnorm(g)
    tol = gtol * (gn if relative else 1.0)
    g2 = float(torch.linalg.vector_norm(g).item())
    g0_2 = g2
    hist = [(J, gn, 0)]
    evals, hvps, it = 1, 0, 0
    Hg = hvp(v, g)
    hvps += 1
    gHg = float(torch.dot(g, Hg).item())
    radius = g2 ** 3 / gHg if gHg > 0.0 else g2
    rejected = 0
    while gn > tol and it < max_iter and rejected < 60:
        eta = min(eta_max, math.sqrt(g2 / max(g0_2, 1e-300)))
        if cg is not None:
            z, Hz, k, boundary = cg(v, g, radius, eta * g2, max_cg)
            hvps += k
        else:
            cnt = [0]

            def hv(w):
                cnt[0] += 1
                return hvp(v, w)

            z, Hz, k, boundary = _cg_steihaug(g, hv, radius, eta * g2, max_cg)
            hvps += cnt[0]
        pred = -(float(torch.dot(g, z).item()) + 0.5 * float(torch.dot(z, Hz).item()))
        v_new = v + z
        J_new, g_new = ev(v_new)
        evals += 1
        J_new = float(J_new)
        zn = float(torch.linalg.vector_norm(z).item())
        rho = (J - J_new) / pred if pred > 0.0 and math.isfinite(J_new) else -1.0
        noise_ok = (math.isfinite(J_new) and J_new <= J + eps_f * abs(J)
                    and _gnorm(g_new) < gn and pred > 0.0 and abs(J - J_new) <= 2 * eps_f * abs(J))
        if rho < 0.25 and not noise_ok:
            radius = 0.25 * zn
        elif rho > 0.75 and boundary:
            radius = min(2.0 * radius, radius_max)
        if rho > 1e-4 or noise_ok:
            v, J, g = v_new, J_new, g_new
            g2 = float(torch.linalg.vector_norm(g).item())
            gn = _gnorm(g)
            it += 1
            rejected = 0
            hist.append((J, gn, k))
        else:
            rejected += 1
    return NewtonResult(v, J, gn, it, evals, hvps, gn <= tol, time.perf_counter() - t0, hist)


def _rotate_yz(v, angle):
    """Rotate the (y, z) components of every node of v by its angle (the map of eq.
    (displacement) composed with v)."""
    V = v.reshape(-1, 3)
    c, s = torch.cos(angle), torch.sin(angle)
    out = V.clone()
    out[:, 1] = c * V[:, 1] + s * V[:, 2]
    out[:, 2] = -s * V[:, 1] + c * V[:, 2]
    return out.reshape(-1)


def torsion_continuation(ev, hvp, coords, dirichlet, *, lx=0.4, T=24, alpha_max=8.0 * math.pi,
                         gtol=1e-9, relative=True, max_iter=1000, cg=None, **newton_kw):
    """Benchmark 4's sequence of minimisations: the bar's right face (x = lx) rotated about the
    x axis by alpha(t) = alpha_max t / T, the left face fixed, t = 1..T, each problem started
    from the previous minimiser (trust-region Newton-CG on the kernels).  The start of step 1
    is the twist of eq. (displacement) with alpha(1); the start of step t > 1 is the previous
    minimiser rotated by the increment alpha_max/T * x/lx (the face values then are exactly
    those of alpha(t)).  Yields (t, NewtonResult).  coords, dirichlet: the mesh's (n, 3) node
    coordinates and per-dof Dirichlet mask, as tensors on the evaluators' device; cg and any
    other keyword (eta_max, max_cg, ...) go to newton_cg."""
    x = coords[:, 0]
    X = coords.reshape(-1)
    fixed = dirichlet.reshape(-1) != 0
    v = _rotate_yz(X, alpha_max / T * x / lx)
    for t in range(1, T + 1):
        if t > 1:
            v = _rotate_yz(v, alpha_max / T * x / lx)
            exact = _rotate_yz(X, alpha_max * t / T * x / lx)
            v = torch.where(fixed, exact, v)
        r = newton_cg(ev, hvp, v, gtol=gtol, relative=relative, max_iter=max_iter, cg=cg, **newton_kw)
        v = r.v
        yield t, r


def mesh_hvp(mesh):
    """hvp(v, w) -> Hw with the library's FP64 Hessian-vector kernel."""
    def hvp(v, w):
        return mesh.hessian_vector(v, w)
    return hvp


def mesh_cg(mesh):
    """cg(v, g, radius, tol, max_cg) for newton_cg: the library's device-resident Steihaug CG
    over the same Hessian-vector kernel."""
    def cg(v, g, radius, tol, max_cg):
        return mesh.cg_steihaug(v, g, radius, tol, max_cg)
    return cg


# ----------------------------------------------------------------------------------------
# Evaluators over the CUDA library
# ----------------------------------------------------------------------------------------

# Relative rounding level of J per element precision: FP64 and double-float sums are accurate
# to about 1e-14 of the energy scale; the FP32 element path to about 1e-7 of it.
EPS_F = {0: 1e-10, 1: 1e-6, 2: 1e-10}


def mesh_evaluator(mesh, gradient: str = "exact", eps: float = 1e-6):
    """ev(v) -> (J, g) with the library's kernels: exact gradient or patch central
    differences (the energy comes from the same call in the exact case).  J is a device
    scalar, read by the caller (float(J)) when it needs it.  ev.eps_f is the
    rounding level of J at the mesh's active precision when the evaluator is made."""
    if gradient == "exact":
        def ev(v):
            J, g = mesh.energy_gradient(v)
            return J, g
    elif gradient == "fd":
        def ev(v):
            J = mesh.energy(v)
            g = mesh.gradient_fd(v, eps)
            return J, g
    else:
        raise ValueError(gradient)
    ev.eps_f = EPS_F.get(mesh.precision, 1e-10)
    return ev


def batch_evaluator(batch, meshes, device=0):
    """batch_eval(list of (k, v)) -> list of (J, g) through one fe_batch call."""
    from . import fem
    dev = torch.device("cuda", device)
    works = []
    for mesh in meshes:
        wb = fem.Batch.work_bytes(mesh)
        buf = torch.empty(wb + 256, dtype=torch.uint8, device=dev)
        off = (-buf.data_ptr()) % 256
        works.append(buf[off: off + wb])

    def batch_eval(trials):
        items, outs = [], []
        for k, v in trials:
            J = torch.empty((), dtype=torch.float64, device=dev)
            g = torch.empty(meshes[k].ndof, dtype=torch.float64, device=dev)
            items.append((meshes[k], v.contiguous(), J, g, works[k]))
            outs.append((J, g))
        batch.run(items)
        batch.sync_status()
        return [(J.item(), g) for J, g in outs]

    return batch_eval


# ----------------------------------------------------------------------------------------
# Nested iteration over uniformly refined meshes
# ----------------------------------------------------------------------------------------

def prolongation_pairs(coarse_coords, coarse_elems, fine_coords):
    """For a fine mesh whose nodes are the coarse nodes and the midpoints of the coarse edges
    (one uniform refinement of P1 simplices), the coarse node pair (a, b) of every fine node:
    the coarse P1 function takes the value (v_a + v_b) / 2 there (a == b at coarse nodes).
    When the fine elements refine the coarse ones, this is the exact injection of the coarse
    space into the fine one.  Returns an int64 array (n_fine, 2); ValueError for a fine node
    that is neither.  Node matching uses coordinates quantised to 2^-20 of the bounding box."""
    cc = np.asarray(coarse_coords, dtype=np.float64)
    ce = np.asarray(coarse_elems, dtype=np.int64)
    fc = np.asarray(fine_coords, dtype=np.float64)
    k = ce.shape[1]
    nc = cc.shape[0]
    edges = np.sort(np.concatenate([ce[:, [i, j]] for i in range(k) for j in range(i + 1, k)]), axis=1)
    ekey = np.unique(edges[:, 0] * nc + edges[:, 1])
    edges = np.stack([ekey // nc, ekey % nc], axis=1)
    own = np.arange(nc, dtype=np.int64)
    pairs = np.concatenate([np.stack([own, own], axis=1), edges])
    pts = np.concatenate([cc, 0.5 * (cc[edges[:, 0]] + cc[edges[:, 1]])])
    lo = np.minimum(pts.min(axis=0), fc.min(axis=0))
    ext = np.maximum(np.maximum(pts.max(axis=0), fc.max(axis=0)) - lo, 1e-300)

    def keys(x):
        q = np.rint((x - lo) / ext * (1 << 20)).astype(np.int64)
        out = np.zeros(x.shape[0], dtype=np.int64)
        for m in range(x.shape[1]):
            out = (out << 21) | q[:, m]
        return out
    kc, kf = keys(pts), keys(fc)
    order = np.argsort(kc, kind="stable")
    pos = np.searchsorted(kc[order], kf)
    pos = np.minimum(pos, len(order) - 1)
    hit = kc[order][pos] == kf
    if not hit.all():
        raise ValueError(f"{int((~hit).sum())} fine nodes are neither coarse nodes nor coarse edge midpoints")
    return pairs[order[pos]]


def prolong(v, pairs, d=1):
    """The coarse P1 function v (d components per node) at the fine nodes given by pairs."""
    idx = torch.as_tensor(pairs, device=v.device)
    V = v.reshape(-1, d)
    return (0.5 * (V[idx[:, 0]] + V[idx[:, 1]])).reshape(-1)


def nested_newton(levels, v0, *, d=1, **newton_kw):
    """Nested iteration: trust-region Newton-CG on each mesh of a uniformly refined sequence,
    the first started from v0 and each later one from the previous minimiser prolonged to it.
    levels: list of (ev, hvp, cg, coords, elems) per mesh, coarse to fine (cg may be None);
    newton_kw go to newton_cg.  Returns the list of NewtonResult."""
    out = []
    v = v0
    prev = None
    for ev, hvp, cg, coords, elems in levels:
        if prev is not None:
            v = prolong(v, prolongation_pairs(prev[0], prev[1], coords), d)
        r = newton_cg(ev, hvp, v, cg=cg, **newton_kw)
        out.append(r)
        v = r.v
        prev = (coords, elems)
    return out
