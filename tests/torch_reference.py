"""Plain PyTorch FP64 restatement of one blended step on a fully periodic grid,
for differentiating the scheme with autograd (test infrastructure only).

It follows the same equations as the oracle -- Maxwellians of the D2Q5 example
(Sec. 2), face states u* (eq. D2Q5_convexproof_3) and dF (eq. 2nd-order_flux),
theta = min(1, theta_rho, theta_p) with the PP density bound (Sec. 3.3.3) and the
internal-energy bound (Sec. 3.4), and the update eq. (blending_u1) / eq.
(blending_u) -- written with whole-array ops and torch.roll, so autograd gives
the transpose of the step independently of the hand-written CUDA adjoint. The
state is a (20, ny, nx) tensor: u, then u_1..u_4 (x+, x-, y+, y-), 4 planes each.
"""
import torch


def fluxes(u, gamma):
    r, m1, m2, E = u[0], u[1], u[2], u[3]
    v1, v2 = m1 / r, m2 / r
    p = (gamma - 1.0) * (E - 0.5 * r * (v1 * v1 + v2 * v2))
    f = torch.stack([m1, m1 * v1 + p, m2 * v1, (E + p) * v1])
    g = torch.stack([m2, m1 * v2, m2 * v2 + p, (E + p) * v2])
    return f, g


def max_speed(u, gamma):
    r = u[0]
    v1, v2 = u[1] / r, u[2] / r
    p = (gamma - 1.0) * (u[3] - 0.5 * r * (v1 * v1 + v2 * v2))
    return float((torch.sqrt(v1 * v1 + v2 * v2) + torch.sqrt(gamma * p / r)).max())


def init_populations(u, a, alpha, gamma):
    f, g = fluxes(u, gamma)
    w = (1.0 - alpha) / 4.0
    return torch.cat([u, w * u + f / (2 * a), w * u - f / (2 * a), w * u + g / (2 * a), w * u - g / (2 * a)])


def theta_pp(us, df, kappa, eps):
    """theta = min(1, theta_rho, theta_p), clamped at 0; us, df: (4, ...). Every
    selection is a torch.where with the comparison and tie rule of the scheme's
    step (1 before theta_rho before theta_p; r1 only where r1 > r2), so autograd
    differentiates the branch the step takes."""
    rs, m1, m2, Es = us[0], us[1], us[2], us[3]
    dr, dm1, dm2, dE = df[0], df[1], df[2], df[3]
    one = torch.ones_like(rs)
    zero = torch.zeros_like(rs)
    adr = torch.abs(dr)
    nz = adr > 0
    t_rho = kappa * rs / torch.where(nz, adr, one) - eps
    th_rho = torch.where(nz, torch.where(t_rho > 0, t_rho, zero), one)
    g0 = m1 * m1 + m2 * m2 - 2.0 * rs * Es
    g1 = 2.0 * (dr * Es + dE * rs - dm1 * m1 - dm2 * m2)
    cq = dm1 * dm1 + dm2 * dm2 - 2.0 * dr * dE
    disc = g1 * g1 - 4.0 * g0 * cq
    pos = disc > 0
    sq = torch.where(pos, torch.sqrt(torch.where(pos, disc, one)), zero)
    inside = (rs > 0) & (g0 < 0)
    r1 = adr / torch.where(inside, rs, one)
    r2 = (torch.abs(g1) + sq) / (-2.0 * torch.where(inside, g0, -one))
    r = torch.where(r1 > r2, r1, r2)
    rpos = r > 0
    t_p = kappa / torch.where(rpos, r, one) - eps
    th_p = torch.where(rpos, torch.where(t_p > 0, t_p, zero), one)
    th_p = torch.where(inside, th_p, zero)
    th = torch.where(th_rho < one, th_rho, one)
    th = torch.where(th_p < th, th_p, th)
    return torch.where(th < 0, zero, th)


def step(s, a, limiter, alpha=0.5, gamma=1.4, eps=1e-16):
    """One step; limiter 0 (theta = 0), 1 (theta = 1) or 2 (PP)."""
    u, P1, P2, P3, P4 = s[0:4], s[4:8], s[8:12], s[12:16], s[16:20]
    f, g = fluxes(u, gamma)
    w = (1.0 - alpha) / 4.0
    kappa = a * (1.0 - alpha) / 2.0
    M1, M2 = w * u + f / (2 * a), w * u - f / (2 * a)
    M3, M4 = w * u + g / (2 * a), w * u - g / (2 * a)
    d1, d2, d3, d4 = M1 - P1, M2 - P2, M3 - P3, M4 - P4
    E = lambda t: torch.roll(t, -1, dims=-1)    # value of the east neighbour
    N = lambda t: torch.roll(t, -1, dims=-2)    # value of the north neighbour
    Wr = lambda t: torch.roll(t, 1, dims=-1)    # value of the west neighbour
    Sr = lambda t: torch.roll(t, 1, dims=-2)    # value of the south neighbour
    # east x-face and north y-face of every cell
    us_x = 0.5 * (u + E(u)) - (E(f) - f) / (2 * kappa)
    df_x = a * (d1 - E(d2))
    us_y = 0.5 * (u + N(u)) - (N(g) - g) / (2 * kappa)
    df_y = a * (d3 - N(d4))
    if limiter == 0:
        tx = torch.zeros_like(u[0])
        ty = torch.zeros_like(u[0])
    elif limiter == 1:
        tx = torch.ones_like(u[0])
        ty = torch.ones_like(u[0])
    else:
        tx = theta_pp(us_x, df_x, kappa, eps)
        ty = theta_pp(us_y, df_y, kappa, eps)
    tE, tW, tN, tS = tx, Wr(tx), ty, Sr(ty)
    P1n = Wr(M1 + tE * d1)          # pulled from the west cell across its east face
    P2n = E(M2 + tW * d2)           # pulled from the east cell across its west face
    P3n = Sr(M3 + tN * d3)
    P4n = N(M4 + tS * d4)
    un = P1n + P2n + P3n + P4n + alpha * u - tW * d2 - tE * d1 - tS * d4 - tN * d3
    return torch.cat([un, P1n, P2n, P3n, P4n])


def rollout(u0, nsteps, a, limiter, alpha=0.5, gamma=1.4, eps=1e-16):
    s = init_populations(u0, a, alpha, gamma)
    for _ in range(nsteps):
        s = step(s, a, limiter, alpha, gamma, eps)
    return s


def speed_max(u, gamma):
    """lambda = max over the cells of |v| + sqrt(gamma p / rho), differentiable (the
    gradient of a max goes to the cell where it is reached)."""
    r = u[0]
    v1, v2 = u[1] / r, u[2] / r
    p = (gamma - 1.0) * (u[3] - 0.5 * r * (v1 * v1 + v2 * v2))
    return (torch.sqrt(v1 * v1 + v2 * v2) + torch.sqrt(gamma * p / r)).max()


def rollout_dynamic(u0, nsteps, limiter, alpha=0.5, gamma=1.4, eps=1e-16):
    """As rollout, with the dynamic kinetic speed of Sec. 4: a^n = 2 lambda(s^n) / (1 - alpha)
    before every step (a^0 from u_0, which also sets the initial populations)."""
    a = 2.0 * speed_max(u0, gamma) / (1.0 - alpha)
    s = init_populations(u0, a, alpha, gamma)
    for _ in range(nsteps):
        s = step(s, a, limiter, alpha, gamma, eps)
        a = 2.0 * speed_max(s[0:4], gamma) / (1.0 - alpha)
    return s
