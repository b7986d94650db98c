"""Plain PyTorch FP64 restatement of one blended step, on a fully periodic grid or
(step_frame) inside a two-layer ghost frame, for differentiating the scheme with
autograd (test infrastructure only).

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


def theta_p_only(us, df, kappa, eps):
    """The internal-energy bound theta_p of Sec. 3.4 (1 where the radius is 0, 0 where
    u* is outside G), with the scheme's tie rules."""
    rs, m1, m2, Es = us[0], us[1], us[2], us[3]
    dr, dm1, dm2, dE = df[0], df[1], df[2], df[3]
    one = torch.ones_like(rs)
    zero = torch.zeros_like(rs)
    adr = torch.abs(dr)
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
    return torch.where(inside, th_p, zero)


def theta_lmp(us, df, mu_l, nu_l, mu_r, nu_r, kappa, eps):
    """theta = min(1, theta_rho LMP, theta_p), clamped at 0: the three cases of
    Sec. 3.3.1 with the bounds of the cells left (l) and right (r) of the face."""
    rs, dr = us[0], df[0]
    one = torch.ones_like(rs)
    zero = torch.zeros_like(rs)
    nz = dr != 0
    a1, a2 = nu_r - rs, rs - mu_l
    b1, b2 = rs - mu_r, nu_l - rs
    dsafe = torch.where(nz, dr, one)
    t_pos = kappa * torch.where(a1 < a2, a1, a2) / dsafe
    t_neg = -kappa * torch.where(b1 < b2, b1, b2) / dsafe
    th_rho = torch.where(nz, torch.where(dr > 0, t_pos, t_neg), one)
    th_p = theta_p_only(us, df, kappa, eps)
    th = torch.where(th_rho < one, th_rho, one)
    th = torch.where(th_p < th, th_p, th)
    return torch.where(th < 0, zero, th)


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
    """One step; limiter 0 (theta = 0), 1 (theta = 1), 2 (PP), 3 (LMP) or 4 (RLMP).
    The LMP bounds of a cell are the min / max of its density and of rho* on its four
    faces (eq. LMP_minmax), in the order rho, west, east, south, north (the gradient
    of a min goes to the first place it is reached); RLMP scales them by 0.999 and
    1.001 (Sec. 3.3.2)."""
    return _core(s, a, limiter, alpha, gamma, eps)


def _core(s, a, limiter, alpha, gamma, eps, sponge_x=None, sponge_y=None):
    """The step on an array whose neighbours are taken with torch.roll: the whole
    grid when it is periodic, or a grid padded with its ghost frame, where the
    values rolled in at the outer edge reach no cell more than two cells inside it
    (the stencil's radius). sponge_x / sponge_y: faces forced to theta = 0."""
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
    elif limiter == 2:
        tx = theta_pp(us_x, df_x, kappa, eps)
        ty = theta_pp(us_y, df_y, kappa, eps)
    else:
        rho_all = torch.stack([u[0], Wr(us_x[0]), us_x[0], Sr(us_y[0]), us_y[0]])
        mu = torch.min(rho_all, dim=0).values
        nu = torch.max(rho_all, dim=0).values
        if limiter == 4:
            mu, nu = 0.999 * mu, 1.001 * nu
        tx = theta_lmp(us_x, df_x, mu, nu, E(mu), E(nu), kappa, eps)
        ty = theta_lmp(us_y, df_y, mu, nu, N(mu), N(nu), kappa, eps)
    if sponge_x is not None:
        tx = torch.where(sponge_x, torch.zeros_like(tx), tx)
        ty = torch.where(sponge_y, torch.zeros_like(ty), ty)
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


def ghost_frame(cfg, a, t=0.0, sponge=0, const_in_a=False):
    """The oracle's ghost fill (two layers, x rule then y rule) as a gather: every
    entry of the padded (20, ny + 4, nx + 4) array is sign x one state entry, or a
    constant (a prescribed state's value, which does not depend on the state). The
    map is read off the oracle by filling a state whose entries are distinct codes
    (and twice those codes: a constant does not change). With sponge = w > 0, the
    faces with theta = 0 of the sponge layer (Sec. 4.2: every face of a cell within
    w cells of a zero-gradient side, ghost cells included; sides of one type).
    const_in_a: also the constants as c0 + c1 / a (a prescribed ghost's populations are
    its Maxwellians, affine in 1 / a), read off fills at a and 2a, for a^n that varies."""
    import numpy as np

    from oracle import oracle as O

    nx, ny = cfg.nx, cfg.ny
    code = (np.arange(20 * ny * nx, dtype=np.float64) + 1.0).reshape(20, ny, nx)
    e1 = O.fill_ghosts(cfg, code, a, t)
    e2 = O.fill_ghosts(cfg, 2.0 * code, a, t)
    const = e2 == e1
    lin = ~const
    if not np.array_equal(e2[lin], 2.0 * e1[lin]):
        raise ValueError("ghost fill is not a signed copy")
    frame = {"src": torch.tensor(np.where(lin, np.abs(e1) - 1.0, 0.0).astype(np.int64)),
             "sign": torch.tensor(np.where(lin, np.sign(e1), 0.0)),
             "cval": torch.tensor(np.where(const, e1, 0.0))}
    if const_in_a:
        e3 = O.fill_ghosts(cfg, code, 2.0 * a, t)
        frame["c1"] = torch.tensor(np.where(const, 2.0 * a * (e1 - e3), 0.0))
        frame["c0"] = torch.tensor(np.where(const, 2.0 * e3 - e1, 0.0))
    if sponge > 0:
        I, J = np.meshgrid(np.arange(-2, nx + 2), np.arange(-2, ny + 2))
        zg = [b == 1 for b in cfg.bc]
        m = (zg[0] & (I < sponge)) | (zg[1] & (I >= nx - sponge)) | (zg[2] & (J < sponge)) | \
            (zg[3] & (J >= ny - sponge))
        frame["sponge_x"] = torch.tensor(m | np.roll(m, -1, axis=1))
        frame["sponge_y"] = torch.tensor(m | np.roll(m, -1, axis=0))
    return frame


def step_frame(s, a, limiter, frame, alpha=0.5, gamma=1.4, eps=1e-16):
    """One step of a grid with a boundary: the ghost frame gathered from s, the step
    on the padded array, its interior returned."""
    cval = frame["c0"] + frame["c1"] / a if "c1" in frame else frame["cval"]
    P = frame["sign"] * s.reshape(-1)[frame["src"]] + cval
    out = _core(P, a, limiter, alpha, gamma, eps, frame.get("sponge_x"), frame.get("sponge_y"))
    return out[:, 2:-2, 2:-2]


def rollout_frame(u0, nsteps, a, limiter, frame, alpha=0.5, gamma=1.4, eps=1e-16):
    s = init_populations(u0, a, alpha, gamma)
    for _ in range(nsteps):
        s = step_frame(s, a, limiter, frame, alpha, gamma, eps)
    return s


def rollout_dynamic_frame(u0, nsteps, limiter, frame, alpha=0.5, gamma=1.4, eps=1e-16, lam_bc=0.0):
    """rollout_dynamic inside a ghost frame; with prescribed states the frame carries
    its constants as functions of a (const_in_a), and lambda^n also covers the
    prescribed states' speed lam_bc (Sec. 4 preamble; cells win a tie)."""
    lb = torch.tensor(lam_bc, dtype=u0.dtype)

    def speed(u):
        sc = speed_max(u, gamma)
        return torch.where(lb > sc, lb, sc)

    a = 2.0 * speed(u0) / (1.0 - alpha)
    s = init_populations(u0, a, alpha, gamma)
    for _ in range(nsteps):
        s = step_frame(s, a, limiter, frame, alpha, gamma, eps)
        a = 2.0 * speed(s[0:4]) / (1.0 - alpha)
    return s
