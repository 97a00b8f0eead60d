"""The candidate set of the block-per-cell platelet sweep, checked on the CPU.

The block kernel (csrc/platelet.cu, k_psweep_staged) tests a trial of a home
platelet against the platelets listed in the 27 cells around the HOME cell,
after a binary32 prefilter of their offsets from the home cell's centre with
a relative margin of 2^-10; Algorithm 5, like the reference, scans the 27
cells around the TRIAL's cell.  Where the kernel applies (stencil half-width
1 and 2 (a + t) + 2^-15 a + 2 c_m below the cell width) both sets hold every
platelet within contact reach, so the contact decision -- an OR over pairs --
is the same.  These tests run sweeps in the reference's order on the kernel
specification's predicate and compare the two decisions for every trial the
reference evaluates; the sweep itself must end where the reference's does."""
import numpy as np
import pytest

import oracle
import plt_kernel_spec as spec
import srm_inputs


def min_image(v, L):
    """Minimum image of difference vectors (rows), as the reference takes it."""
    v = np.array(v, dtype=float)
    v = np.where(v > 0.5 * L, v - L, v)
    return np.where(v < -0.5 * L, v + L, v)


def emulate_sweep(w, lam, c_m, c_r):
    """One sweep in the canonical order; returns (X, U, trials compared)."""
    L = np.asarray(w.box, dtype=float)
    X, U = w.x.copy(), w.u.copy()
    a, t = lam * w.a0, lam * w.t0
    n, wc = oracle.grid(3, w.box, lam, w.a0 + w.t0, c_m)
    n, wc = np.asarray(n, dtype=np.int64), np.asarray(wc, dtype=float)
    # the kernel's conditions
    assert all(2.0 * (a + t) + 2.0 * c_m < wc)
    assert all(2.0 * (a + t) + a * 2.0 ** -15 + 2.0 * c_m < wc)
    cell3 = np.floor(X / wc).astype(np.int64) % n
    lin = cell3[:, 0] + n[0] * (cell3[:, 1] + n[1] * cell3[:, 2])
    members = {}
    for i in np.argsort(lin, kind="stable"):
        members.setdefault(int(lin[i]), []).append(int(i))

    def around(c):
        out = []
        for sx in (-1, 0, 1):
            for sy in (-1, 0, 1):
                for sz in (-1, 0, 1):
                    e = (c + np.array([sx, sy, sz])) % n
                    out += members.get(int(e[0] + n[0] * (e[1] + n[1] * e[2])), [])
        return np.asarray(out, dtype=np.int64)

    reach64 = 2.0 * (a + t) * 1.001  # beyond it the specification's first test is false

    def decide(ids, q, u):
        return any(spec.collide32(min_image(X[j] - q, L), u, U[j], a, t) for j in ids)

    def contact(cands, q, u, pid):
        cands = cands[cands != pid]
        d = min_image(X[cands] - q, L)
        return decide(cands[np.einsum("ij,ij->i", d, d) <= reach64 * reach64], q, u)

    af, tf = np.float32(a), np.float32(t)
    rf = np.float32((np.float32(af + af) + np.float32(np.float32(tf + tf) + af * np.float32(2.0 ** -16)))
                    * np.float32(1.0 + 2.0 ** -10))
    Lf = L.astype(np.float32)

    def staged_contact(cands, centre, q, u, pid):
        cands = cands[cands != pid]
        qf = min_image(q - centre, L).astype(np.float32)
        v = min_image(X[cands] - centre, L).astype(np.float32) - qf
        v = np.where(v > Lf / 2, v - Lf, v)
        v = np.where(v < -Lf / 2, v + Lf, v).astype(np.float32)
        d2 = (v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]).astype(np.float32) + v[:, 2] * v[:, 2]
        return decide(cands[d2 <= rf * rf], q, u)

    compared = 0
    for chi in range(27):
        for cz in range(chi // 9, n[2], 3):
            for cy in range((chi // 3) % 3, n[1], 3):
                for cx in range(chi % 3, n[0], 3):
                    home = np.array([cx, cy, cz])
                    cell = int(cx + n[0] * (cy + n[1] * cz))
                    staged = around(home)
                    centre = (home + 0.5) * wc
                    for pid in members.get(cell, []):
                        x0, u0 = X[pid].copy(), U[pid].copy()
                        for l in range(10):
                            q, u = oracle.plt_trial(w.seed, 0, pid, l, w.box, c_m, c_r, x0, u0)
                            qc = np.floor(q / wc).astype(np.int64) % n
                            A = contact(around(qc), q, u, pid)
                            B = staged_contact(staged, centre, q, u, pid)
                            assert A == B, (pid, l)
                            compared += 1
                            if not A:
                                X[pid], U[pid] = q, u
                                break
    return X, U, compared


@pytest.mark.parametrize("scale,c_m_rel,c_r", [(2.5, 0.05, 0.05), (2.2, 0.1, 0.1)])
def test_staged_set_decides_as_the_trial_stencil(scale, c_m_rel, c_r):
    w = srm_inputs.platelets(seed=17, n=700, aspect=20.0, rho_t=3.0)
    lam = scale * w.lambda0
    c_m = c_m_rel * w.extra["D"]
    X, U, compared = emulate_sweep(w, lam, c_m, c_r)
    assert compared > 700
    o = oracle.PlateletSystem(w.box, w.x, w.u, w.a0, w.t0, lam=lam, lam_t=1.0, seed=w.seed, c_w=w.c_w, c_m=c_m,
                              c_r=c_r, contact=spec.address())
    o.sweep()
    ox, ou = o.state()
    np.testing.assert_array_equal(X, ox)
    np.testing.assert_array_equal(U, ou)
