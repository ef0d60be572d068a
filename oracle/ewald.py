"""Plain FP64 CPU oracle of the ionic-melt forces (test infrastructure only:
the test suite, the smoke check and the CPU legs of ``bench.py`` use it; the
GPU library never does).

What it computes, for point charges q_i in a periodic cubic box of side L
with a short-range Buckingham pair potential (arXiv 2503.07526 Sec. 2.3 and
Sec. 5.3 for the SPME method, Appendix B for the per-particle split; the
Ewald and SPME formulas follow Essmann et al., J. Chem. Phys. 103, 8577
(1995), whose notation Appendix B uses):

  U = sum_{i<j, r<rc} [A exp(-r/rho) - C/r^6 + ke q_i q_j erfc(alpha r)/r]
      + E_rec - ke alpha/sqrt(pi) sum_i q_i^2,
  E_rec = ke/(2 pi V) sum_{m != 0} exp(-pi^2 m^2/alpha^2)/m^2 |S(m)|^2,
  S(m) = sum_j q_j exp(2 pi i m.r_j),  m = n/L for integer vectors n.

Per-particle quantities split every term to its particles: a pair term half
to each partner; the self term to its particle; the reciprocal energy as
E_j = ke/(2 pi V) sum_m g(m) q_j Re[exp(2 pi i m.r_j) S(m)*] (these sum to
E_rec), and the reciprocal virial with the same weights times the tensor
delta_ab - 2 (1 + pi^2 m^2/alpha^2) m_a m_b / m^2 (these sum to the total
reciprocal virial).  The per-particle virial of a pair term is
1/2 r_ij (x) f_ij, as for Lennard-Jones.

Two reciprocal evaluators: ``ewald_reciprocal`` is the plain k-space sum
above; ``spme_reciprocal`` is the smooth particle-mesh Ewald approximation
of it (cardinal B-splines of order n, Euler exponential splines b(m), a
K^3 mesh and numpy's FFT), with the per-particle energy and virial read off
the mesh as Appendix B describes: the particle's spline weights times the
mesh convolved with the same k-space kernels.

Pins (tests/test_oracle_ewald.py): the Madelung constant of rock salt; the
independence of the Ewald total from alpha; forces and the virial against
finite differences of the energy; SPME against the plain k-space sum as the
mesh and the order grow; per-particle sums against totals.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

KE = 14.399645478425668  # e^2 / (4 pi eps0) in eV Angstrom


def cell_matrix(L):
    """The box as a 3x3 matrix whose columns are the lattice vectors: a
    cubic side L, three orthorhombic sides, or a matrix (used to strain the
    box in the tests)."""
    L = np.asarray(L, dtype=np.float64)
    if L.ndim == 0:
        return np.eye(3) * float(L)
    if L.ndim == 1:
        return np.diag(L)
    return L


def _min_image(d, h):
    hinv = np.linalg.inv(h)
    s = hinv @ d
    return h @ (s - np.round(s))


def real_space(r, q, L, *, A, rho, C, alpha, rc, ke=KE):
    """Short-range part: Buckingham plus the real-space Ewald term, all
    pairs with r < rc under the minimum image (rc below half the shortest
    box height).  r [3, n]; L a side, three sides or a cell matrix.
    Returns (F [3, n], E [n], W [6, n], U) with W in xx yy zz xy xz yz."""
    h = cell_matrix(L)
    n = r.shape[1]
    F = np.zeros((3, n))
    E = np.zeros(n)
    W = np.zeros((6, n))
    U = 0.0
    c2 = 2.0 * alpha / math.sqrt(math.pi)
    for i in range(n - 1):
        d = _min_image(r[:, i:i + 1] - r[:, i + 1:], h)  # r_i - r_j
        rr = np.sqrt((d * d).sum(axis=0))
        m = rr < rc
        d, rr = d[:, m], rr[m]
        qq = ke * q[i] * q[i + 1:][m]
        ex = A * np.exp(-rr / rho)
        u = ex - C / rr ** 6 + qq * erfc(alpha * rr) / rr
        dudr = -ex / rho + 6.0 * C / rr ** 7 - qq * (erfc(alpha * rr) / rr ** 2 + c2 * np.exp(-(alpha * rr) ** 2) / rr)
        fpair = -dudr / rr * d  # force on i from j
        js = np.nonzero(m)[0] + i + 1
        F[:, i] += fpair.sum(axis=1)
        np.add.at(F, (slice(None), js), -fpair)
        E[i] += 0.5 * u.sum()
        np.add.at(E, js, 0.5 * u)
        w = 0.5 * np.stack([d[0] * fpair[0], d[1] * fpair[1], d[2] * fpair[2],
                            d[0] * fpair[1], d[0] * fpair[2], d[1] * fpair[2]])
        W[:, i] += w.sum(axis=1)
        np.add.at(W, (slice(None), js), w)
        U += u.sum()
    return F, E, W, U


def self_energy(q, alpha, ke=KE):
    """Per-particle Ewald self term -ke alpha/sqrt(pi) q_i^2."""
    return -ke * alpha / math.sqrt(math.pi) * np.asarray(q, dtype=np.float64) ** 2


def _kernel(m2, alpha):
    return np.exp(-(math.pi ** 2) * m2 / alpha ** 2) / m2


def _virial_tensor(mv, m2, alpha):
    """delta_ab - 2 (1 + pi^2 m^2/alpha^2) m_a m_b / m^2 for the six
    components xx yy zz xy xz yz; mv [3, ...], m2 [...]."""
    fac = 2.0 * (1.0 + math.pi ** 2 * m2 / alpha ** 2) / m2
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    return np.stack([(1.0 if a == b else 0.0) - fac * mv[a] * mv[b] for a, b in pairs])


def ewald_reciprocal(r, q, L, *, alpha, nmax, ke=KE):
    """Plain k-space sum over reciprocal vectors m = h^-T n for integer n
    with 0 < |n|_inf <= nmax (h the cell matrix; m = n/L for a cube).
    Returns (F [3, n], E [n], W [6, n], E_rec, W_rec [6])."""
    h = cell_matrix(L)
    V = abs(float(np.linalg.det(h)))
    g = np.arange(-nmax, nmax + 1)
    nx, ny, nz = np.meshgrid(g, g, g, indexing="ij")
    nv = np.stack([nx.ravel(), ny.ravel(), nz.ravel()]).astype(np.float64)
    keep = np.any(nv != 0, axis=0)
    mv = np.linalg.inv(h).T @ nv[:, keep]  # [3, M]
    m2 = (mv * mv).sum(axis=0)
    gk = _kernel(m2, alpha)
    phase = 2.0 * math.pi * (mv.T @ r)  # [M, n]
    ez = np.exp(1j * phase)
    S = ez @ q  # [M]
    pref = ke / (2.0 * math.pi * V)
    contrib = (ez * np.conj(S)[:, None]).real  # Re[e^{2 pi i m r_j} S*]
    E = pref * q * (gk[:, None] * contrib).sum(axis=0)
    Fm = (ez * np.conj(S)[:, None]).imag  # Im[e^{2 pi i m r_j} S*]
    F = 2.0 * ke / V * q[None, :] * (mv @ (gk[:, None] * Fm))
    T = _virial_tensor(mv, m2, alpha)  # [6, M]
    W = pref * q[None, :] * ((T * gk[None, :]) @ contrib)
    Erec = pref * float((gk * np.abs(S) ** 2).sum())
    Wrec = pref * (T * (gk * np.abs(S) ** 2)[None, :]).sum(axis=1)
    return F, E, W, Erec, Wrec


def bspline(u, n):
    """Cardinal B-spline M_n(u) (support [0, n]) by the recursion
    M_n(u) = u/(n-1) M_{n-1}(u) + (n-u)/(n-1) M_{n-1}(u-1), M_2 the hat."""
    u = np.asarray(u, dtype=np.float64)
    if n == 2:
        return np.where((u >= 0) & (u <= 2), 1.0 - np.abs(u - 1.0), 0.0)
    return (u * bspline(u, n - 1) + (n - u) * bspline(u - 1.0, n - 1)) / (n - 1)


def bspline_moduli(K, n):
    """|b(m)|^2 = 1 / |sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k/K)|^2."""
    k = np.arange(n - 1)
    Mk = bspline(k + 1.0, n)
    m = np.arange(K)
    den = np.abs(np.exp(2j * math.pi * np.outer(m, k) / K) @ Mk) ** 2
    return 1.0 / den


def spme_reciprocal(r, q, L, *, alpha, K, order, ke=KE, virial="derivative"):
    """Smooth particle-mesh Ewald on a K^3 mesh with order-n splines
    (K >= order) in a cubic box of side L.  Returns (F [3, n], E [n],
    W [6, n], E_rec, W_rec [6]) like ewald_reciprocal.

    The per-particle virial: with virial="derivative" (Appendix B's form),
    W_ab,j = delta_ab E_j minus the m_a m_b term, whose factor m_a m_b is
    carried by two derivatives of the particle's spline weights,
    m_a m_b exp(2 pi i m.r) ~ (K/(2 pi i L))^2 b(m) sum_k d_a d_b W_j(k) ...,
    applied to one more convolved mesh psi (kernel B C h with
    h = 2 (1 + pi^2 m^2/alpha^2)/m^2).  With virial="tensor", six meshes
    convolved with the full tensor kernel are read with the plain weights.
    Both tend to the k-space sum's per-particle virial."""
    L = float(L)
    if K < order:
        raise ValueError("the mesh must have at least `order` points per side")
    n_at = r.shape[1]
    V = L ** 3
    u = np.mod(r / L, 1.0) * K  # scaled fractional coordinates [3, n]
    # spline weights and derivatives on the n mesh points k = floor(u) - t, t = 0..n-1
    base = np.floor(u).astype(np.int64)
    t = np.arange(order)
    w = np.zeros((3, n_at, order))
    dw = np.zeros((3, n_at, order))
    d2w = np.zeros((3, n_at, order))
    for a in range(3):
        x = (u[a] - base[a])[:, None] + t[None, :]  # argument u - k
        w[a] = bspline(x, order)
        dw[a] = bspline(x, order - 1) - bspline(x - 1.0, order - 1)
        d2w[a] = bspline(x, order - 2) - 2.0 * bspline(x - 1.0, order - 2) + bspline(x - 2.0, order - 2)
    idx = np.mod(base[:, :, None] - t[None, None, :], K)  # [3, n, order]
    # charge mesh Q(k)
    Q = np.zeros((K, K, K))
    for j in range(n_at):
        blk = q[j] * np.einsum("a,b,c->abc", w[0, j], w[1, j], w[2, j])
        Q[np.ix_(idx[0, j], idx[1, j], idx[2, j])] += blk
    # k-space kernels
    mi = np.fft.fftfreq(K, d=1.0 / K)  # 0, 1, ..., -1
    mx, my, mz = np.meshgrid(mi, mi, mi, indexing="ij")
    mv = np.stack([mx, my, mz]) / L
    m2 = (mv * mv).sum(axis=0)
    m2[0, 0, 0] = 1.0
    bm = bspline_moduli(K, order)
    B = bm[:, None, None] * bm[None, :, None] * bm[None, None, :]
    Ck = _kernel(m2, alpha) / (math.pi * V)
    Ck[0, 0, 0] = 0.0
    FQ = np.fft.fftn(Q)
    BC = B * Ck
    Erec = 0.5 * ke * float((BC * np.abs(FQ) ** 2).sum())
    T = _virial_tensor(mv, m2, alpha)
    T[:, 0, 0, 0] = 0.0
    Wrec = 0.5 * ke * (T * (BC * np.abs(FQ) ** 2)[None]).sum(axis=(1, 2, 3))
    # convolved meshes: theta * Q = IFFT(B C FFT(Q)) (times K^3 for numpy's IFFT scaling)
    phi = np.fft.ifftn(BC * FQ).real * K ** 3
    if virial == "tensor":
        phiW = [np.fft.ifftn(BC * T[c] * FQ).real * K ** 3 for c in range(6)]
    elif virial == "derivative":
        hk = 2.0 * (1.0 + math.pi ** 2 * m2 / alpha ** 2) / m2
        psi = np.fft.ifftn(BC * hk * FQ).real * K ** 3
    else:
        raise ValueError("virial must be 'derivative' or 'tensor'")
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    cw = ke * (K / L) ** 2 / (8.0 * math.pi ** 2)
    F = np.zeros((3, n_at))
    E = np.zeros(n_at)
    W = np.zeros((6, n_at))
    for j in range(n_at):
        sub = np.ix_(idx[0, j], idx[1, j], idx[2, j])
        P = phi[sub]
        wj = np.einsum("a,b,c->abc", w[0, j], w[1, j], w[2, j])
        E[j] = 0.5 * ke * q[j] * float((wj * P).sum())
        if virial == "tensor":
            for c in range(6):
                W[c, j] = 0.5 * ke * q[j] * float((wj * phiW[c][sub]).sum())
        else:
            Psi = psi[sub]
            for c, (a, b) in enumerate(pairs):
                f = [w[0, j], w[1, j], w[2, j]]
                if a == b:
                    f[a] = d2w[a, j]
                else:
                    f[a], f[b] = dw[a, j], dw[b, j]
                S = float((np.einsum("a,b,c->abc", *f) * Psi).sum())
                W[c, j] = (E[j] if a == b else 0.0) + cw * q[j] * S
        g0 = np.einsum("a,b,c->abc", dw[0, j], w[1, j], w[2, j])
        g1 = np.einsum("a,b,c->abc", w[0, j], dw[1, j], w[2, j])
        g2 = np.einsum("a,b,c->abc", w[0, j], w[1, j], dw[2, j])
        F[:, j] = -ke * q[j] * (K / L) * np.array([(g0 * P).sum(), (g1 * P).sum(), (g2 * P).sum()])
    return F, E, W, Erec, Wrec


def rock_salt(cells, a):
    """Ions of a rock-salt crystal of cubic lattice constant a (cells^3 unit
    cells, 8 ions each): positions [3, n], charges +1 / -1, box side."""
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.arange(cells)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    org = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], 1).astype(np.float64)
    cat = (org[:, None, :] + base[None]).reshape(-1, 3)
    an = (org[:, None, :] + base[None] + np.array([0.5, 0, 0])).reshape(-1, 3)
    pos = np.concatenate([cat, an]) * a + 0.25 * a
    q = np.concatenate([np.ones(len(cat)), -np.ones(len(an))])
    return np.ascontiguousarray(pos.T), q, cells * a


def total_energy(r, q, L, *, A, rho, C, alpha, rc, nmax=None, K=None, order=None, ke=KE):
    """Total potential energy with the plain k-space sum (nmax) or SPME (K,
    order)."""
    _, _, _, Ur = real_space(r, q, L, A=A, rho=rho, C=C, alpha=alpha, rc=rc, ke=ke)
    if nmax is not None:
        Erec = ewald_reciprocal(r, q, L, alpha=alpha, nmax=nmax, ke=ke)[3]
    else:
        Erec = spme_reciprocal(r, q, L, alpha=alpha, K=K, order=order, ke=ke)[3]
    return Ur + Erec + self_energy(q, alpha, ke).sum()
