"""Closed-form linear wake of a weak bi-Gaussian electron driver (test pin for the oracle).

Derived from the paper's model (Eqs. 1-7) in the weak-driver limit n_b/n_p << 1 of a cold
plasma, with a conducting wall at r = R (psi(R) = 0).  For n_b = n0 rho(r) f(xi),
rho = exp(-r^2 / 2 sigma_r^2):

    g(xi)  = int_0^xi sin(xi - s) f(s) ds,   g'(xi) = int_0^xi cos(xi - s) f(s) ds
    H(r)   = int_0^R G_R(r, s) rho(s) s ds,  (lap_perp - 1) H = -rho,  H(R) = 0
    G_R    = I0(r<) [K0(r>) - K0(R) I0(r>) / I0(R)]
    psi    = n0 g H,   E_z = n0 g' H,   B_theta = n0 f H',   E_r = n0 (f - g) H'

(the textbook linear PWFA result; the source is truncated to xi >= 0 like the box).
"""
import numpy as np
from scipy import integrate, special


def radial_profiles(r_nodes, sigma_r, R):
    i0R, k0R = special.i0(R), special.k0(R)
    rho = lambda s: np.exp(-s * s / (2 * sigma_r ** 2))

    def kern_in(s):   # s > r: I0(r) [K0(s) - K0(R) I0(s)/I0(R)]
        return special.k0(s) - k0R * special.i0(s) / i0R

    H = np.zeros(len(r_nodes))
    Hp = np.zeros(len(r_nodes))
    opts = dict(epsabs=1e-14, epsrel=1e-12, limit=400)
    for n, r in enumerate(r_nodes):
        if r >= R:
            H[n] = 0.0
        # inner part s < r: G = I0(s) [K0(r) - K0(R) I0(r)/I0(R)]
        inner = integrate.quad(lambda s: special.i0(s) * rho(s) * s, 0, r, **opts)[0] if r > 0 else 0.0
        outer = integrate.quad(lambda s: kern_in(s) * rho(s) * s, r, R, **opts)[0] if r < R else 0.0
        H[n] = (special.k0(r) - k0R * special.i0(r) / i0R) * inner + special.i0(r) * outer if r > 0 else outer
        if r > 0:
            Hp[n] = (-special.k1(r) - k0R * special.i1(r) / i0R) * inner + special.i1(r) * outer
    return H, Hp


def longitudinal_profiles(xi_nodes, xi_d, sigma_z):
    f = lambda s: np.exp(-0.5 * ((s - xi_d) / sigma_z) ** 2)
    g = np.zeros(len(xi_nodes))
    gp = np.zeros(len(xi_nodes))
    opts = dict(epsabs=1e-14, epsrel=1e-12, limit=400)
    for n, x in enumerate(xi_nodes):
        if x > 0:
            g[n] = integrate.quad(lambda s: np.sin(x - s) * f(s), 0, x, **opts)[0]
            gp[n] = integrate.quad(lambda s: np.cos(x - s) * f(s), 0, x, **opts)[0]
    return f(np.asarray(xi_nodes)), g, gp


def linear_fields(cfg):
    """psi, ez, bth, er on the (nxi+1) x (nr+1) nodes of cfg (single bunch, n_w = 0)."""
    r = np.arange(cfg.nr + 1) * (cfg.rmax / cfg.nr)
    xi = np.arange(cfg.nxi + 1) * (cfg.ximax / cfg.nxi)
    H, Hp = radial_profiles(r, cfg.sigma_r, cfg.rmax)
    f, g, gp = longitudinal_profiles(xi, cfg.xi_d, cfg.sigma_zd)
    n0 = cfg.n_d
    return {"psi": n0 * np.outer(g, H), "ez": n0 * np.outer(gp, H),
            "bth": n0 * np.outer(f, Hp), "er": n0 * np.outer(f - g, Hp)}


# ---------------------------------------------------------------------------------------
# slab geometry (x, xi), mirror plane x = 0, conducting wall at x = L
# ---------------------------------------------------------------------------------------
# (d_x^2 - 1) H = -rho on 0 <= x <= L with H'(0) = 0 (even) and H(L) = 0:
#   H(x) = int_0^L G(x, s) rho(s) ds,  G = cosh(x<) sinh(L - x>) / cosh(L),
# and the same linear fields psi = n0 g H, E_z = n0 g' H, B_y = n0 f H', E_x = n0 (f - g) H'.
def slab_profiles(x_nodes, sigma, L):
    rho = lambda s: np.exp(-s * s / (2 * sigma ** 2))
    cL = np.cosh(L)
    H = np.zeros(len(x_nodes))
    Hp = np.zeros(len(x_nodes))
    opts = dict(epsabs=1e-14, epsrel=1e-12, limit=400)
    for n, x in enumerate(x_nodes):
        inner = integrate.quad(lambda s: np.cosh(s) * rho(s), 0, x, **opts)[0] if x > 0 else 0.0   # s < x
        outer = integrate.quad(lambda s: np.sinh(L - s) * rho(s), x, L, **opts)[0] if x < L else 0.0  # s > x
        H[n] = (np.sinh(L - x) * inner + np.cosh(x) * outer) / cL
        Hp[n] = (-np.cosh(L - x) * inner + np.sinh(x) * outer) / cL
    return H, Hp


def slab_linear_fields(cfg):
    """psi, ez, bth (B_y), er (E_x) on the (nxi+1) x (nr+1) nodes of a slab cfg."""
    x = np.arange(cfg.nr + 1) * (cfg.rmax / cfg.nr)
    xi = np.arange(cfg.nxi + 1) * (cfg.ximax / cfg.nxi)
    H, Hp = slab_profiles(x, cfg.sigma_r, cfg.rmax)
    f, g, gp = longitudinal_profiles(xi, cfg.xi_d, cfg.sigma_zd)
    n0 = cfg.n_d
    return {"psi": n0 * np.outer(g, H), "ez": n0 * np.outer(gp, H),
            "bth": n0 * np.outer(f, Hp), "er": n0 * np.outer(f - g, Hp)}
