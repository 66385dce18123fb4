"""A NumPy model of the D2Q9 step in the deviation variables g = f - W rho0, with FP32 or
FP64 arithmetic (test infrastructure; it shares no code with the CUDA path or the oracle).

It exists to study how FP32 rounding drives the result away from the FP64 oracle over many
steps. It follows the Appendix steps 1-9 in the same variables as the kernels:
  step 1   fbar+ = g + b1 (geq - g) + c1 S at the cells (eq. f_bar_+, increment form);
  step 2   ghosts: periodic images, or 2 f0 - f1 at walls (x first, then y);
  steps 3-4 interface values 1/2 (L + R) - kappa e_d (R - L) - kappa e_t dC/4 (eq. gradient,
           cross-point tangential differences);
  step 5   NEQ velocity walls (eq. NEQ) with x_c the boundary cell's opposite interface;
  steps 6-7 interface moments (weight h/2 on G) and f = F + b7 (geq - F) + c7 S;
  steps 8-9 g' = fbar+ + (fbar+ - g)/3 - dt c/dx sum_d e_d (f_d+ - f_d-).
Lattice units: dx = 1, RT = 1/3 (c = 1), rho0 = 1. Domains: periodic in x with NEQ walls in
y (the channel), or NEQ walls on all four sides with a moving +y lid (the cavity).

`cell="one_rounding"` replaces the FP32 cell stage by a form with one rounding at the scale
of the equilibrium's odd term: moments by compensated (two-sum) summation, e.m kept as an
exact two-term sum, the small terms of W (q + 3 e.m) added first and a single fused
multiply-add with 3W last, and the relaxation itself as one fused multiply-add.
`cell="lean"` is its cheaper form: only the momentum sums compensated, e.m a single rounded
value, the odd term still one final fused multiply-add with 3W.
`cell="moments_only"` / `"equilibrium_only"` apply one half of it (the other half as in the
kernels: plain sums; e.m rounded, then fma(e.m, 3, q) and W x)."""
import numpy as np

F32, F64 = np.float32, np.float64
E = np.array([(ex, ey) for ex in (-1, 0, 1) for ey in (-1, 0, 1)])
_W1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
WT = np.array([_W1[ex] * _W1[ey] for ex, ey in E])
EX = E[:, 0].astype(F64)[:, None, None]
EY = E[:, 1].astype(F64)[:, None, None]
WB = WT[:, None, None]


def _geq(d, mx, my, T):
    """Deviation equilibrium of eq. icfeq: W (drho + 3 e.m + 4.5 (e.m)^2 - 1.5 m.m)."""
    em = (EX * mx[None] + EY * my[None]).astype(T)
    mm = (mx * mx + my * my).astype(T)
    x = d[None] + T(3) * em + T(4.5) * em * em - T(1.5) * mm[None]
    return (WB.astype(T) * x).astype(T)


def _moments(g, Gx, Gy, w, T):
    """drho = sum g, m = sum e g + rho0 G w (units of c)."""
    d = g.sum(axis=0, dtype=T).astype(T)
    mx = ((EX.astype(T) * g).sum(axis=0, dtype=T) + T(w) * T(Gx)).astype(T)
    my = ((EY.astype(T) * g).sum(axis=0, dtype=T) + T(w) * T(Gy)).astype(T)
    return d, mx, my


def _relax(g, d, mx, my, Gx, Gy, b, c, T):
    """g + b (geq - g) + c S, S = 3 (e - u).G f_eq (eq. S in these units)."""
    ge = _geq(d, mx, my, T)
    v = g + T(b) * (ge - g)
    if Gx or Gy:
        eG = (EX * Gx + EY * Gy).astype(T)
        Gm = (T(Gx) * mx + T(Gy) * my).astype(T)
        v = v + T(c) * T(3) * (eG - Gm[None]) * (WB.astype(T) + ge)
    return v.astype(T)


def _fma(a, b, c):
    """Fused multiply-add of FP32 operands: the exact product and sum, rounded once (the
    FP64 sum of an exact FP32 x FP32 product and an FP32 addend rounds to nearest; the rare
    double rounding is immaterial here)."""
    return (np.asarray(a, F64) * np.asarray(b, F64) + np.asarray(c, F64)).astype(F32)


def _two_sum(a, b):
    """s + e == a + b exactly (Knuth's TwoSum)."""
    s = (a + b).astype(F32)
    bb = (s - a).astype(F32)
    return s, ((a - (s - bb)) + (b - bb)).astype(F32)


def _csum(terms):
    """Compensated sum of FP32 arrays, rounded once."""
    s = np.zeros_like(terms[0])
    c = np.zeros_like(terms[0])
    for t in terms:
        s, e = _two_sum(s, t.astype(F32))
        c = (c + e).astype(F32)
    return (s + c).astype(F32)


_W3 = 3.0 * WT
_W3H = _W3.astype(F32)
_W3L = (_W3 - _W3H.astype(F64)).astype(F32)
_WH = WT.astype(F32)
_WL = (WT - _WH.astype(F64)).astype(F32)


def _nsum(terms):
    """Plain left-to-right FP32 sum."""
    s = np.zeros_like(terms[0])
    for t in terms:
        s = (s + t.astype(F32)).astype(F32)
    return s


def _cell_one_rounding(g, Gx, Gy, b1, c1, dt, compensated=True, one_rounding=True, lean=False):
    """The FP32 cell stage with compensated moments and/or the one-rounding equilibrium
    (otherwise: plain sums, and e.m rounded, fma(e.m, 3, q) and W x as in the kernels).
    lean: only the momentum sums compensated, and e.m a single rounded value."""
    w = dt / 2
    sm = _csum if compensated else _nsum
    d = (_nsum if lean else sm)([g[k] for k in range(9)])
    mx = sm([F32(E[k, 0]) * g[k] for k in range(9) if E[k, 0]] + [np.full_like(g[0], F32(w) * F32(Gx))])
    my = sm([F32(E[k, 1]) * g[k] for k in range(9) if E[k, 1]] + [np.full_like(g[0], F32(w) * F32(Gy))])
    mm = _fma(mx, mx, (my * my).astype(F32))
    base = _fma(F32(-1.5), mm, d)                     # drho - 1.5 m.m (small)
    ge = np.empty_like(g)
    for k in range(9):
        a, b = (F32(E[k, 0]) * mx).astype(F32), (F32(E[k, 1]) * my).astype(F32)
        if one_rounding:
            emh, eml = _two_sum(a, b) if not lean else ((a + b).astype(F32), np.zeros_like(a))
            q = _fma((F32(4.5) * emh).astype(F32), emh, base)  # even part (small)
            small = (_WH[k] * q + _WL[k] * q + _W3L[k] * emh + _W3H[k] * eml).astype(F32)
            ge[k] = _fma(_W3H[k], emh, small)                 # the one rounding at the odd term's scale
        else:
            em = (a + b).astype(F32)
            x = _fma(em, F32(3), _fma((F32(4.5) * em).astype(F32), em, base))
            ge[k] = _fma(_WL[k], x, (_WH[k] * x).astype(F32))
    v = _fma(F32(b1), (ge - g).astype(F32), g)
    if Gx or Gy:
        eG = (EX * Gx + EY * Gy).astype(F32)
        Gm = (F32(Gx) * mx + F32(Gy) * my).astype(F32)
        v = _fma((F32(c1) * F32(3) * (eG - Gm[None])).astype(F32), (WB.astype(F32) + ge).astype(F32), v)
    return v


class Model:
    """D2Q9 channel (xwalls=False) or cavity (xwalls=True, lid speed on +y), from rest."""

    def __init__(self, nx, ny, nu, T=F64, G=(0.0, 0.0), dt=0.5, xwalls=False, lid=0.0, cell="plain"):
        self.nx, self.ny, self.nu, self.T, self.G, self.dt = nx, ny, nu, T, G, dt
        self.xwalls, self.lid, self.cell = xwalls, lid, cell
        self.g = np.zeros((9, ny, nx), dtype=T)

    def _neq(self, F, Fc, sel, uw, T):
        """Step 5, eq. NEQ, for a velocity wall of speed (uw, 0): the incoming velocities take
        f_eq(rho_c, u_w) + F(x_c) - f_eq(rho_c, u_c), with x_c's interface moments."""
        h = self.dt / 2
        d, cx, cy = _moments(Fc, self.G[0], self.G[1], h / 2, T)
        za = np.zeros_like(cx)
        v = Fc + _geq(d, za + T(uw), za, T) - _geq(d, cx, cy, T)
        F[sel] = v[sel]

    def step(self):
        T, (Gx, Gy), dt, nx, ny = self.T, self.G, self.dt, self.nx, self.ny
        tau, h = self.nu * 3.0, dt / 2
        b1, c1 = 3 * h / (2 * tau + dt), 3 * tau * h / (2 * tau + dt)
        b7, c7 = h / (2 * tau + h), tau * h / (2 * tau + h)
        g = self.g
        if self.cell != "plain" and T == F32:
            fp = _cell_one_rounding(g, Gx, Gy, b1, c1, dt, compensated=self.cell != "equilibrium_only",
                                    one_rounding=self.cell != "moments_only", lean=self.cell == "lean")
        else:
            d, mx, my = _moments(g, Gx, Gy, dt / 2, T)
            fp = _relax(g, d, mx, my, Gx, Gy, b1, c1, T)
        x = np.zeros((9, ny + 2, nx + 2), dtype=T)   # step 2
        x[:, 1:-1, 1:-1] = fp
        if self.xwalls:
            x[:, 1:-1, 0] = T(2) * x[:, 1:-1, 1] - x[:, 1:-1, 2]
            x[:, 1:-1, -1] = T(2) * x[:, 1:-1, -2] - x[:, 1:-1, -3]
        else:
            x[:, 1:-1, 0], x[:, 1:-1, -1] = fp[:, :, -1], fp[:, :, 0]
        x[:, 0] = T(2) * x[:, 1] - x[:, 2]
        x[:, -1] = T(2) * x[:, -2] - x[:, -3]
        k, q4 = T(h), T(0.25)                        # kappa = h c / dx
        L, R = x[:, 1:-1, :-1], x[:, 1:-1, 1:]
        Fx = T(0.5) * (L + R) - k * EX.astype(T) * (R - L) \
            - k * EY.astype(T) * q4 * ((x[:, 2:, :-1] + x[:, 2:, 1:]) - (x[:, :-2, :-1] + x[:, :-2, 1:]))
        L, R = x[:, :-1, 1:-1], x[:, 1:, 1:-1]
        Fy = T(0.5) * (L + R) - k * EY.astype(T) * (R - L) \
            - k * EX.astype(T) * q4 * ((x[:, :-1, 2:] + x[:, 1:, 2:]) - (x[:, :-1, :-2] + x[:, 1:, :-2]))
        Fx, Fy = Fx.astype(T), Fy.astype(T)
        Fx0 = Fx.copy()
        for j, jc, s, uw in ((0, 1, 1, 0.0), (ny, ny - 1, -1, self.lid)):
            row = Fy[:, j:j + 1, :]
            self._neq(row, Fy[:, jc:jc + 1, :], (E[:, 1] * s > 0), uw, T)
        if self.xwalls:
            for i, ic, s in ((0, 1, 1), (nx, nx - 1, -1)):
                col = Fx[:, :, i:i + 1]
                self._neq(col, Fx0[:, :, ic:ic + 1], (E[:, 0] * s > 0), 0.0, T)
        fx, fy = (_relax(F, *_moments(F, Gx, Gy, h / 2, T), Gx, Gy, b7, c7, T) for F in (Fx, Fy))
        acc = EX.astype(T) * (fx[:, :, 1:] - fx[:, :, :-1]) + EY.astype(T) * (fy[:, 1:] - fy[:, :-1])
        self.g = (fp + (fp - g) / T(3) - T(dt) * acc).astype(T)

    def velocity(self):
        g = self.g.astype(F64)
        return np.stack([((EX * g).sum(axis=0) + self.G[0] * self.dt / 2).ravel(),
                         ((EY * g).sum(axis=0) + self.G[1] * self.dt / 2).ravel()])
