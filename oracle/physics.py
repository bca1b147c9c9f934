"""Pointwise physics of the compressible Navier-Stokes equations (oracle).

Test infrastructure only.  Follows Sec. 2 of the paper:

* state U = (rho, rho*u_1..rho*u_d, rho*E), E = e_i + |u|^2/2, e_i = c_v theta;
* convective flux F^c_i = (rho u_i, rho u_i u_j + p delta_ij, rho u_i H),
  H = E + p/rho  (Eq. of the inviscid and viscous fluxes);
* ideal gas p = rho R theta, R = c_p - c_v;
* viscous flux F^nu_i = (0, tau_ij, tau_ij u_j - q_i) with
  tau_ij = mu (d_i u_j + d_j u_i) + lambda (div u) delta_ij, lambda = -2 mu / 3,
  q_i = -kappa d_i theta, kappa = c_p mu / Pr, mu constant.

Nondimensionalisation (the paper only says "aerodynamic reference values"):
rho_ref = |u_ref| = L_ref = 1 and theta_inf = 1, hence R = 1/(gamma Ma^2),
c_v = R/(gamma-1), c_p = gamma c_v, mu = 1/Re.  Then kappa/c_v = gamma mu / Pr
and Ma drops out of the operator.

Gradients are of the conservative variables (Q = grad U), converted to
velocity and temperature gradients by the chain rule.

The convective numerical flux is local Lax-Friedrichs (Rusanov), which the
paper does not use (it uses the Vijayasundaram flux); the wave speed is
max over both sides of |u.n| + c.  ``absr``/``maxr`` branch on real parts so
that every function here is complex-step differentiable; at a tie max picks
the interior (minus) side, and d|x|/dx at 0 is 0.

Tensor layout: the field axis is axis 1 (U[k][nf][...]); direction axes
(``Sn``, ``Q``) sit right after the element axis.
"""
import torch


def absr(x):
    return x * torch.sign(x.real).to(x.dtype)


def maxr(a, b):
    return torch.where(a.real >= b.real, a, b)


class Gas:
    def __init__(self, gamma, Re=0.0, Pr=0.72, viscous=False):
        self.gamma = float(gamma)
        self.viscous = bool(viscous)
        self.mu = (1.0 / Re) if (viscous and Re > 0) else 0.0
        self.Pr = float(Pr)
        self.lam = -2.0 * self.mu / 3.0
        # kappa / c_v = gamma * mu / Pr (Ma-independent, see module doc)
        self.k_over_cv = self.gamma * self.mu / self.Pr


def primitives(U, gas, d):
    rho = U[:, 0]
    m = U[:, 1:1 + d]
    rE = U[:, d + 1]
    u = m / rho.unsqueeze(1)
    ke = 0.5 * (m * u).sum(1)
    p = (gas.gamma - 1.0) * (rE - ke)
    return rho, u, p, rE


def convective_flux(U, gas, d):
    """F^c[k][i][field][...] for directions i."""
    rho, u, p, rE = primitives(U, gas, d)
    F = []
    for i in range(d):
        comps = [rho * u[:, i]]
        for j in range(d):
            comps.append(rho * u[:, i] * u[:, j] + (p if i == j else 0.0))
        comps.append((rE + p) * u[:, i])
        F.append(torch.stack(comps, 1))
    return torch.stack(F, 1)


def normal_convective_flux(U, Sn, gas, d):
    """F^c(U) . Sn  with Sn[k][d][...] -> [k][nf][...]."""
    F = convective_flux(U, gas, d)
    return sum(F[:, i] * Sn[:, i].unsqueeze(1) for i in range(d))


def sound_speed(U, gas, d):
    rho, u, p, _ = primitives(U, gas, d)
    return torch.sqrt(gas.gamma * p / rho)


def llf_flux(UL, UR, Sn, gas, d):
    """Local Lax-Friedrichs flux through the area-weighted normal Sn (own side = L).

    F* = 1/2 (F(UL) + F(UR)).Sn - 1/2 lam (UR - UL),
    lam = max(|uL.Sn| + cL |Sn|, |uR.Sn| + cR |Sn|).
    """
    sJ = torch.sqrt(sum(Sn[:, i] * Sn[:, i] for i in range(d)))
    _, uL, _, _ = primitives(UL, gas, d)
    _, uR, _, _ = primitives(UR, gas, d)
    unL = sum(uL[:, i] * Sn[:, i] for i in range(d))
    unR = sum(uR[:, i] * Sn[:, i] for i in range(d))
    lam = maxr(absr(unL) + sound_speed(UL, gas, d) * sJ, absr(unR) + sound_speed(UR, gas, d) * sJ)
    FL = normal_convective_flux(UL, Sn, gas, d)
    FR = normal_convective_flux(UR, Sn, gas, d)
    return 0.5 * (FL + FR) - 0.5 * lam.unsqueeze(1) * (UR - UL)


def velocity_temperature_gradients(U, Q, gas, d):
    """From Q[k][a][field][...] = d U_field / d x_a: grad u[k][a][i], grad e_i[k][a].

    d_a u_i = (d_a m_i - u_i d_a rho) / rho,
    d_a e   = (d_a (rho E) - E d_a rho) / rho - u_j d_a u_j   (e = internal energy / mass).
    """
    rho, u, p, rE = primitives(U, gas, d)
    Et = rE / rho
    gu = torch.stack([torch.stack([(Q[:, a, 1 + i] - u[:, i] * Q[:, a, 0]) / rho for i in range(d)], 1)
                      for a in range(d)], 1)                                   # [k][a][i]
    ge = torch.stack([(Q[:, a, d + 1] - Et * Q[:, a, 0]) / rho
                      - sum(u[:, j] * gu[:, a, j] for j in range(d)) for a in range(d)], 1)
    return u, gu, ge


def stress(gu, gas, d):
    div = sum(gu[:, i, i] for i in range(d))
    tau = [[gas.mu * (gu[:, i, j] + gu[:, j, i]) + (gas.lam * div if i == j else 0.0)
            for j in range(d)] for i in range(d)]
    return tau


def viscous_flux(U, Q, gas, d):
    """F^nu[k][i][field][...]."""
    u, gu, ge = velocity_temperature_gradients(U, Q, gas, d)
    tau = stress(gu, gas, d)
    F = []
    for i in range(d):
        q_i = -gas.k_over_cv * ge[:, i]
        comps = [torch.zeros_like(tau[i][0])]
        comps += [tau[i][j] for j in range(d)]
        comps.append(sum(tau[i][j] * u[:, j] for j in range(d)) - q_i)
        F.append(torch.stack(comps, 1))
    return torch.stack(F, 1)


def normal_viscous_flux(U, Q, Sn, gas, d):
    F = viscous_flux(U, Q, gas, d)
    return sum(F[:, i] * Sn[:, i].unsqueeze(1) for i in range(d))


def wall_state(U, d):
    """No-slip wall state U_w = (rho, 0, .., 0, rho e_i) (App. B, no-slip state)."""
    rho = U[:, 0]
    m = U[:, 1:1 + d]
    rei = U[:, d + 1] - 0.5 * (m * m).sum(1) / rho
    zeros = [torch.zeros_like(rho)] * d
    return torch.stack([rho] + zeros + [rei], 1)


def mirror_state(U, Sn, d):
    """Reflected state (rho, m - 2 (m.n) n, rho E) used as the LLF ghost at walls."""
    sJ2 = sum(Sn[:, i] * Sn[:, i] for i in range(d))
    mn = sum(U[:, 1 + i] * Sn[:, i] for i in range(d)) / sJ2
    comps = [U[:, 0]] + [U[:, 1 + i] - 2.0 * mn * Sn[:, i] for i in range(d)] + [U[:, d + 1]]
    return torch.stack(comps, 1)


def adiabatic_wall_viscous_flux(U, Q, Sn, gas, d):
    """F^{nu,w}(U_w, Q).Sn with q.n = 0: (0, tau(U_w, Q).Sn, 0) since u_w = 0."""
    Uw = wall_state(U, d)
    u, gu, ge = velocity_temperature_gradients(Uw, Q, gas, d)
    tau = stress(gu, gas, d)
    comps = [torch.zeros_like(U[:, 0])]
    for j in range(d):
        comps.append(sum(tau[i][j] * Sn[:, i] for i in range(d)))
    comps.append(torch.zeros_like(U[:, 0]))
    return torch.stack(comps, 1)


# ---------------------------------------------------------------------------
# Characteristic splitting of the normal inviscid Jacobian (Sec. 3.2) and the
# numerical fluxes built on it (Sec. 3.3, App. B.1.1).
#
# A_n = A_i n_i = P Lambda P^{-1} with eigenvalues u.n - c|n|, u.n (d-fold),
# u.n + c|n| for the (area-weighted) normal n.  With r_k, l_k the right and
# left eigenvectors (l_k r_m = delta_km), P Lambda^{+-} P^{-1} =
# sum_k lambda_k^{+-} r_k l_k^T.  The d-fold eigenvalue's eigenvectors are
# combined through their spectral projector I - r_- l_-^T - r_+ l_+^T (the
# sum of all r_k l_k^T is the identity), so only the two acoustic pairs are
# written out (unit normal nh = n/|n|, enthalpy H = (rho E + p)/rho):
#   r_+- = (1, u +- c nh, H +- c u.nh),
#   l_+- = ((gamma-1)|u|^2/2 -+ c u.nh, -(gamma-1) u +- c nh, gamma-1) / (2 c^2).
# ---------------------------------------------------------------------------

def posr(x):
    """max(x, 0), branching on the real part (complex-step differentiable).
    At x = 0 exactly, where max(x, 0) has no derivative, the value is 0 and
    the derivative the mean of the one-sided ones, 1/2 (through x/2): the
    same convention as d|x|/dx(0) = 0 in max(x, 0) = (x + |x|)/2."""
    return torch.where(x.real > 0, x, torch.where(x.real < 0, torch.zeros_like(x), 0.5 * x))


def negr(x):
    """min(x, 0), branching on the real part; derivative 1/2 at x = 0 exactly."""
    return torch.where(x.real < 0, x, torch.where(x.real > 0, torch.zeros_like(x), 0.5 * x))


def acoustic_eigenvectors(U, Sn, gas, d):
    """Eigenvalues (lam_minus, lam_0, lam_plus) of A_n for the area normal Sn
    and the acoustic eigenvector pairs (r_-, l_-), (r_+, l_+) ([k][nf] each)."""
    rho, u, p, rE = primitives(U, gas, d)
    g = gas.gamma
    sJ = torch.sqrt(sum(Sn[:, i] * Sn[:, i] for i in range(d)))
    nh = Sn / sJ.unsqueeze(1)
    c = torch.sqrt(g * p / rho)
    H = (rE + p) / rho
    un = sum(u[:, i] * nh[:, i] for i in range(d))
    q2 = sum(u[:, i] * u[:, i] for i in range(d))
    r, l = {}, {}
    for s in (-1.0, 1.0):
        r[s] = torch.stack([torch.ones_like(rho)] + [u[:, i] + s * c * nh[:, i] for i in range(d)]
                           + [H + s * c * un], 1)
        l[s] = torch.stack([0.5 * (g - 1.0) * q2 - s * c * un]
                           + [-(g - 1.0) * u[:, i] + s * c * nh[:, i] for i in range(d)]
                           + [torch.full_like(rho, g - 1.0)], 1) / (2.0 * c * c).unsqueeze(1)
    lam = ((un - c) * sJ, un * sJ, (un + c) * sJ)
    return lam, r, l


def split_jacobian(U, Sn, gas, d):
    """A_n^+ and A_n^- ([k][nf][nf]) at state U for the area normal Sn: the
    eigen-splitting P Lambda^{+-} P^{-1} of Sec. 3.2 written with spectral
    projectors (see the block comment above)."""
    lam, r, l = acoustic_eigenvectors(U, Sn, gas, d)
    nf = d + 2
    Pm = r[-1.0].unsqueeze(2) * l[-1.0].unsqueeze(1)
    Pp = r[1.0].unsqueeze(2) * l[1.0].unsqueeze(1)
    I = torch.eye(nf, dtype=U.dtype).expand(U.shape[0], nf, nf)
    P0 = I - Pm - Pp
    out = []
    for part in (posr, negr):
        out.append(part(lam[0])[:, None, None] * Pm + part(lam[1])[:, None, None] * P0
                   + part(lam[2])[:, None, None] * Pp)
    return out[0], out[1]


def vijayasundaram_flux(Uown, Unb, Sn, gas, d):
    """F*_n = A_n^+(Ubar) U_own + A_n^-(Ubar) U_nb with Ubar = (U_own + U_nb)/2
    (Sec. 3.3, Eq. upwinding_Vijayasundaram_sdg), through the area normal Sn
    (own side outward)."""
    Ubar = 0.5 * (Uown + Unb)
    Ap, Am = split_jacobian(Ubar, Sn, gas, d)
    return (Ap @ Uown.unsqueeze(2)).squeeze(2) + (Am @ Unb.unsqueeze(2)).squeeze(2)


def farfield_boundary_state(U, Uinf, Sn, gas, d):
    """U_Gamma of App. B.1.1: A_n(U) U_Gamma = A_n^+(U) U + A_n^-(U) U_inf, i.e.
    the characteristic components with lambda_k >= 0 (outgoing, and the
    undetermined lambda_k = 0) taken from the interior state U, those with
    lambda_k < 0 from the free stream U_inf; eigen-quantities at U."""
    lam, r, l = acoustic_eigenvectors(U, Sn, gas, d)
    nf = d + 2
    Pm = r[-1.0].unsqueeze(2) * l[-1.0].unsqueeze(1)
    Pp = r[1.0].unsqueeze(2) * l[1.0].unsqueeze(1)
    I = torch.eye(nf, dtype=U.dtype).expand(U.shape[0], nf, nf)
    P0 = I - Pm - Pp

    def out_ind(x):
        return (x.real >= 0).to(U.dtype)[:, None, None]
    Pout = out_ind(lam[0]) * Pm + out_ind(lam[1]) * P0 + out_ind(lam[2]) * Pp
    return Uinf + (Pout @ (U - Uinf).unsqueeze(2)).squeeze(2)


def adiabatic_viscous_flux(U, Q, Sn, gas, d):
    """F^{nu,w}[k][i][field] = K_w(U) grad U (App. B.1.2): the viscous flux with the
    normal component of the heat flux removed (q.n = 0 for the unit normal of Sn)."""
    u, gu, ge = velocity_temperature_gradients(U, Q, gas, d)
    sJ2 = sum(Sn[:, i] * Sn[:, i] for i in range(d))
    gn = sum(ge[:, i] * Sn[:, i] for i in range(d)) / sJ2
    ge = ge - gn.unsqueeze(1) * Sn
    tau = stress(gu, gas, d)
    F = []
    for i in range(d):
        comps = [torch.zeros_like(tau[i][0])]
        comps += [tau[i][j] for j in range(d)]
        comps.append(sum(tau[i][j] * u[:, j] for j in range(d)) + gas.k_over_cv * ge[:, i])
        F.append(torch.stack(comps, 1))
    return torch.stack(F, 1)
