"""The potential validation of Sec. 6.3 (Table ValidPotSubs) on the GPU: a homogeneously charged
sphere in a 256^3 domain whose walls carry the analytic potential (per-cell Dirichlet values),
shifted to where its subsampling factor maps the volume worst, solved in
FP64; the relative error e_rPhi = (Phi* - Phi)/Phi over the whole domain is compared with the
published table (tests/golden/valid_pot_errors.txt).

Readings: the L2 norm is the root mean square of e_rPhi over all cells; the maximum norm is the
signed value of largest magnitude. The paper's shift set for the maximal volume-mapping error is
not given; an 11^3 grid over +-0.51 cell / s_f is searched, which finds a different position for
most rows (the volume errors differ), so the checks are the properties every row of the table
shows, the paper's stated bound, the exact agreement of rows with equal s_f R, and the row whose
volume error we reproduce (R = 9, s_f = 1: 1.91 %), value by value.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1410_6609_gb300.solver import Poisson  # noqa: E402

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(__file__)
N = 256


def _max_volume_error_shift(R, sf, npts=11):
    m = int(2 * R + 8)
    V = 4.0 / 3.0 * np.pi * R ** 3
    g = np.linspace(-0.51 / sf, 0.51 / sf, npts)
    best = None
    for dx in g:
        for dy in g:
            for dz in g:
                c = np.array([[m / 2 + dx, m / 2 + dy, m / 2 + dz]])
                e = (oracle.sphere_density((m, m, m), 1.0, c, [R], [1.0], sf).sum() - V) / V
                if best is None or abs(e) > abs(best[0]):
                    best = (e, np.array([dx, dy, dz]))
    return best


def _analytic(r, R, Q):
    """Sec. 6.3: Q/(4 pi eps r) outside, Q/(8 pi eps R) (3 - r^2/R^2) inside (eps = 1)."""
    return torch.where(r >= R, Q / (4 * np.pi * r.clamp_min(1e-300)), Q / (8 * np.pi * R) * (3 - (r / R) ** 2))


def _potential_errors(R, sf):
    e_v, shift = _max_volume_error_shift(R, sf)
    c = np.full(3, N / 2) + shift
    Q = 4.0 / 3.0 * np.pi * R ** 3  # density 1
    cc = torch.arange(N, dtype=torch.float64, device="cuda") + 0.5
    P = Poisson((N, N, N), h=1.0, bc_type=(0,) * 6, bc_value=(0.0,) * 6)
    L = float(N)
    walls = []
    for face in range(6):
        a, side = divmod(face, 2)
        pos = L if side else 0.0
        if a == 0:  # [nz, ny]
            r = torch.sqrt((pos - c[0]) ** 2 + (cc[None, :] - c[1]) ** 2 + (cc[:, None] - c[2]) ** 2)
        elif a == 1:  # [nz, nx]
            r = torch.sqrt((cc[None, :] - c[0]) ** 2 + (pos - c[1]) ** 2 + (cc[:, None] - c[2]) ** 2)
        else:  # [ny, nx]
            r = torch.sqrt((cc[None, :] - c[0]) ** 2 + (cc[:, None] - c[1]) ** 2 + (pos - c[2]) ** 2)
        walls.append(_analytic(r, R, Q).contiguous())
    for face, v in enumerate(walls):
        P.set_bc_field(face, v)
    dev = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64)).cuda()
    rho = P.sphere_density(dev(c[None, :]), dev([R]), dev([1.0]), sf)
    P.set_rhs(rho)
    P.set_solution(None)
    _, rel = P.solve(1e-10, 100)
    assert rel < 1e-10
    phi = P.solution()
    r = torch.sqrt((cc[None, None, :] - c[0]) ** 2 + (cc[None, :, None] - c[1]) ** 2 + (cc[:, None, None] - c[2]) ** 2)
    e = (phi - _analytic(r, R, Q)) / _analytic(r, R, Q)
    l2 = float(torch.sqrt((e * e).mean()))
    emax = float(e.reshape(-1)[int(torch.argmax(e.abs()))])
    P.close()
    return 100 * e_v, 100 * l2, 100 * emax


def test_charged_sphere_potential_against_table():
    table = {(int(r[0]), int(r[1])): r[2:] for r in np.loadtxt(os.path.join(HERE, "golden", "valid_pot_errors.txt"))}
    ours = {key: _potential_errors(*key) for key in [(4, 1), (4, 2), (8, 1), (8, 2), (9, 1)]}
    for (R, sf), (ev, l2, mx) in ours.items():
        # every row of the table: the error follows the mapped charge, |max| >= |e_rVmax|, same sign
        assert np.sign(mx) == np.sign(ev) and abs(mx) >= abs(ev), (R, sf, ev, l2, mx)
        # the paper reports L2 norms below 2 % for every sphere size and subsampling factor
        assert l2 < 2.0
    # equal s_f R map equal volumes (exactly), hence nearly equal potential errors, as the table
    # shows for (4,2)/(8,1)
    assert ours[(4, 2)][0] == ours[(8, 1)][0]
    assert ours[(4, 2)][1:] == pytest.approx(ours[(8, 1)][1:], rel=0.05)
    assert tuple(table[(4, 2)][1:]) == tuple(table[(8, 1)][1:])
    # the row whose maximal volume error we reproduce: its potential errors within 25 %
    ev, l2, mx = ours[(9, 1)]
    t_ev, t_l2, t_mx = table[(9, 1)]
    assert ev == pytest.approx(t_ev, abs=0.01)
    assert l2 == pytest.approx(t_l2, rel=0.25) and mx == pytest.approx(t_mx, rel=0.25)


def _force_errors(R, sfp, rho0=1e-6):
    """e_rFC for force subsampling 1, 2, 3 of a sphere at the potential subsampling's maximal
    volume-error shift, in the homogeneous field of Sec. 6.3 (x walls at 0 and -10, Neumann
    elsewhere); also the volume errors of the three force subsamplings at that position. The
    sphere's force on itself (nonzero when the charge is mapped with another subsampling than the
    force) grows with the charge squared, the applied force with the charge: a small density keeps
    it far below the table's resolution (6e-4 of the applied force at density 1e-3)."""
    _, shift = _max_volume_error_shift(R, sfp)
    c = np.full(3, N / 2) + shift
    Q = rho0 * 4.0 / 3.0 * np.pi * R ** 3
    Fa = Q * 10.0 / N  # E = -(-10 - 0) / L along +x
    P = Poisson((N, N, N), h=1.0, bc_type=(0, 0, 1, 1, 1, 1), bc_value=(0.0, -10.0, 0.0, 0.0, 0.0, 0.0))
    dev = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64)).cuda()
    rho = P.sphere_density(dev(c[None, :]), dev([R]), dev([rho0]), sfp)
    P.set_rhs(rho)
    P.set_solution(None)
    _, rel = P.solve(1e-10, 100)
    assert rel < 1e-10
    m = int(2 * R + 8)
    V = 4.0 / 3.0 * np.pi * R ** 3
    local = np.array([m / 2, m / 2, m / 2]) + shift
    out, ev = [], []
    for sff in (1, 2, 3):
        F = P.force_gather(dev(c[None, :]), dev([R]), dev([rho0]), sff).cpu().numpy()[0]
        out.append(100 * (F[0] - Fa) / Fa)
        ev.append(100 * (oracle.sphere_density((m, m, m), 1.0, local[None, :], [R], [1.0], sff).sum() - V) / V)
        assert abs(F[1]) < 1e-6 * abs(Fa) and abs(F[2]) < 1e-6 * abs(Fa)
    P.close()
    return np.array(out), np.array(ev)


def test_coulomb_force_against_table():
    """Table ValidClmbForceSubs_PotMaxErr (Sec. 6.3): the force error equals the volume-mapping
    error of the force subsampling at the sphere's position (the applied field is exact between
    the plates and the sphere's own force vanishes by symmetry to within 0.01 %), so the diagonal
    (equal subsampling factors) is the potential table's e_rVmax; the row whose position we
    reproduce (R = 9, s_f = 1) matches the paper's 1.91 %."""
    table = {(int(r[0]), int(r[1])): r[2:] for r in np.loadtxt(os.path.join(HERE, "golden", "valid_clmb_force.txt"))}
    pot = {(int(r[0]), int(r[1])): r[2] for r in np.loadtxt(os.path.join(HERE, "golden", "valid_pot_errors.txt"))}
    for R, sfp in [(4, 1), (4, 2), (6, 1), (8, 2), (9, 1), (12, 1)]:
        e_f, e_v = _force_errors(R, sfp)
        assert np.abs(e_f - e_v).max() < 0.01, (R, sfp, e_f, e_v)
        # the paper's own table: its diagonal equals its potential table's e_rVmax
        assert table[(R, sfp)][sfp - 1] == pot[(R, sfp)]
        # subsampling the force more finely than the charge reduces its error
        assert abs(e_f[2]) < abs(e_f[0]) or abs(e_f[0]) < 0.5
    e_f, _ = _force_errors(9, 1)
    assert e_f[0] == pytest.approx(table[(9, 1)][0], abs=0.01)
