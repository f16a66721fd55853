"""Dense-matrix assembly of D_S, D_W, D_B and their free-field symbols.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  This file is the second,
independent route to the operators: it never calls the C oracle.  It builds
colour-space hop matrices H_mu (block (x, x+mu) = V_mu(x)), uses
H_{-mu} = H_mu^dagger for the backward hops, and assembles each operator as a
sum of Kronecker products with the spin matrices.

  Sec. 3     D_S = sum_mu 1/2 E_mu (H_mu - H_mu^+) + m,   E_mu = diag(eta_mu(x))
  def_wils   D_W = sum_mu gamma_mu (x) 1/2 (H_mu - H_mu^+)
                   - 1/2 (-8 + sum_mu (H_mu + H_mu^+)) + m0
  def_bril   D_B = sum_mu gamma_mu (x) grad_mu^iso - 1/2 lap^bri + m0
             grad_mu^iso = sum_{dir: dir_mu != 0} rho_k dir_mu H_dir
             lap^bri     = lambda_0 + sum_{dir != 0} lambda_k H_dir
  Tab. tab:off-axis: the k!-path average obeys the recursion
             H_dir = (1/k) sum_{hops a of dir} H_a H_{dir - a}
             (first hop a, then the average over the orderings of the rest).

Index order of the dense matrices: (site, spin, colour), site lexicographic
s = x + Nx (y + Ny (z + Nz t)), which is the C-order flattening of the
canonical psi[t,z,y,x,v,spin,colour] for one right-hand side v.
"""
from __future__ import annotations

import itertools

import numpy as np

RHO = np.array([0.0, 64.0, 16.0, 4.0, 1.0]) / 432.0        # def_der coefficients
LAMBDA = np.array([-240.0, 8.0, 4.0, 2.0, 1.0]) / 64.0      # def_lap coefficients


def gammas() -> list[np.ndarray]:
    """Euclidean chiral basis: gamma_k = [[0, -i s_k], [i s_k, 0]], gamma_4 = [[0, 1], [1, 0]]."""
    s = [np.array([[0, 1], [1, 0]], dtype=complex),
         np.array([[0, -1j], [1j, 0]], dtype=complex),
         np.array([[1, 0], [0, -1]], dtype=complex)]
    z = np.zeros((2, 2), dtype=complex)
    g = [np.block([[z, -1j * sk], [1j * sk, z]]) for sk in s]
    g.append(np.block([[z, np.eye(2)], [np.eye(2), z]]))
    return g


def gamma5() -> np.ndarray:
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def _lat(V):
    Nt, Nz, Ny, Nx = V.shape[:4]
    return (Nx, Ny, Nz, Nt), V.shape[-1]


def _site(L, x):
    Nx, Ny, Nz, Nt = L
    return (x[0] % Nx) + Nx * ((x[1] % Ny) + Ny * ((x[2] % Nz) + Nz * (x[3] % Nt)))


def _coords(L):
    Nx, Ny, Nz, Nt = L
    t, z, y, x = np.meshgrid(np.arange(Nt), np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1)   # [site, mu]


def hop_matrix(V, mu: int) -> np.ndarray:
    """H_mu with block (x, x+mu) = V_mu(x); shape (vol Nc, vol Nc)."""
    L, Nc = _lat(V)
    vol = int(np.prod(L))
    X = _coords(L)
    Vf = V.reshape(vol, 4, Nc, Nc)
    H = np.zeros((vol, Nc, vol, Nc), dtype=complex)
    for s in range(vol):
        xp = X[s].copy()
        xp[mu] += 1
        H[s, :, _site(L, xp), :] += Vf[s, mu]
    return H.reshape(vol * Nc, vol * Nc)


def _spin_kron(S: np.ndarray, A: np.ndarray, vol: int, Nc: int) -> np.ndarray:
    """F[(x,s,a),(y,t,b)] = S[s,t] A[(x,a),(y,b)]."""
    Ns = S.shape[0]
    A4 = A.reshape(vol, Nc, vol, Nc)
    F = np.einsum("st,xayb->xsaytb", S, A4)
    return F.reshape(vol * Ns * Nc, vol * Ns * Nc)


def dirs_all():
    """All 80 nonzero offsets in {-1,0,1}^4, ordered by hop count."""
    out = [d for d in itertools.product((-1, 0, 1), repeat=4) if any(d)]
    out = [tuple(d[i] for i in range(4)) for d in out]
    return sorted(out, key=lambda d: sum(abs(c) for c in d))


def hop_matrices_W(V) -> dict:
    """H_dir for all 80 dir by the recursion H_dir = (1/k) sum_a H_a H_{dir-a}."""
    H = {}
    for mu in range(4):
        e = [0, 0, 0, 0]
        e[mu] = 1
        Hm = hop_matrix(V, mu)
        H[tuple(e)] = Hm
        e[mu] = -1
        H[tuple(e)] = Hm.conj().T
    for d in dirs_all():
        k = sum(abs(c) for c in d)
        if k == 1:
            continue
        acc = None
        for mu in range(4):
            if d[mu] == 0:
                continue
            a = [0, 0, 0, 0]
            a[mu] = d[mu]
            rest = list(d)
            rest[mu] = 0
            term = H[tuple(a)] @ H[tuple(rest)]
            acc = term if acc is None else acc + term
        H[d] = acc / k
    return H


def W_from_hops(H: dict, V) -> np.ndarray:
    """Read W_dir(x) back out of the hop matrices: [t,z,y,x,81,Nc,Nc] (dir 40 = 1)."""
    L, Nc = _lat(V)
    vol = int(np.prod(L))
    X = _coords(L)
    out = np.zeros((vol, 81, Nc, Nc), dtype=complex)
    for d, Hd in H.items():
        idx = sum((d[m] + 1) * 3 ** m for m in range(4))
        H4 = Hd.reshape(vol, Nc, vol, Nc)
        for s in range(vol):
            out[s, idx] = H4[s, :, _site(L, X[s] + np.array(d)), :]
    out[:, 40] = np.eye(Nc)
    return out.reshape(V.shape[:4] + (81, Nc, Nc))


def dense(op: str, V, mass: float) -> np.ndarray:
    """The dense matrix of D for one right-hand side, order (site, spin, colour).

    mass: staggered m; Wilson / Brillouin m0."""
    L, Nc = _lat(V)
    vol = int(np.prod(L))
    n = vol * Nc
    I = np.eye(n, dtype=complex)
    if op == "staggered":
        X = _coords(L)
        D = mass * I
        for mu in range(4):
            eta = (-1.0) ** X[:, :mu].sum(axis=1)
            E = np.repeat(eta, Nc)
            Hm = hop_matrix(V, mu)
            D = D + 0.5 * E[:, None] * (Hm - Hm.conj().T)
        return D
    g = gammas()
    one = np.eye(4, dtype=complex)
    if op == "wilson":
        D = _spin_kron(one, (4.0 + mass) * I, vol, Nc)
        for mu in range(4):
            Hm = hop_matrix(V, mu)
            D = D + _spin_kron(g[mu], 0.5 * (Hm - Hm.conj().T), vol, Nc)
            D = D - 0.5 * _spin_kron(one, Hm + Hm.conj().T, vol, Nc)
        return D
    if op == "brillouin":
        H = hop_matrices_W(V)
        lap = LAMBDA[0] * I
        nab = [np.zeros((n, n), dtype=complex) for _ in range(4)]
        for d, Hd in H.items():
            k = sum(abs(c) for c in d)
            lap = lap + LAMBDA[k] * Hd
            for mu in range(4):
                if d[mu]:
                    nab[mu] = nab[mu] + RHO[k] * d[mu] * Hd
        D = _spin_kron(one, mass * I - 0.5 * lap, vol, Nc)
        for mu in range(4):
            D = D + _spin_kron(g[mu], nab[mu], vol, Nc)
        return D
    raise ValueError(op)


def dense_apply(D: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a dense D to every right-hand side of a canonical psi."""
    Nv = psi.shape[4]
    vol = int(np.prod(psi.shape[:4]))
    p = psi.reshape(vol, Nv, -1).transpose(1, 0, 2).reshape(Nv, -1)
    o = (D @ p.T).T
    return o.reshape(Nv, vol, -1).transpose(1, 0, 2).reshape(psi.shape)


# ---- free-field symbols (V = 1), a = 1, p_mu = 2 pi n_mu / L_mu --------------

def free_symbol(op: str, p, mass: float) -> np.ndarray:
    """Closed-form momentum-space D(p) for unit links (spin matrix, or 1x1).

    Wilson:    m0 + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu
    Brillouin: m0 + 2 (1 - prod_mu cos^2(p_mu/2))
                  + i sum_mu gamma_mu sin p_mu prod_{nu != mu} (2 + cos p_nu) / 27
    Both follow from the position-space definitions by summing the plane wave
    over the stencil (the rho_k and lambda_k weights factorise per axis).
    The staggered symbol is not translation invariant by one site; its
    checkable closed form is -D_S^2 = sum_mu sin^2 p_mu on plane waves (m = 0).
    """
    p = np.asarray(p, dtype=float)
    g = gammas()
    if op == "wilson":
        D = (mass + np.sum(1 - np.cos(p))) * np.eye(4, dtype=complex)
        for mu in range(4):
            D = D + 1j * np.sin(p[mu]) * g[mu]
        return D
    if op == "brillouin":
        c2 = np.prod(np.cos(p / 2) ** 2)
        D = (mass + 2 * (1 - c2)) * np.eye(4, dtype=complex)
        for mu in range(4):
            s = np.sin(p[mu]) * np.prod([2 + np.cos(p[nu]) for nu in range(4) if nu != mu]) / 27.0
            D = D + 1j * s * g[mu]
        return D
    raise ValueError(op)


def momenta(L):
    """All lattice momenta p = 2 pi n / L (periodic)."""
    axes = [2 * np.pi * np.arange(n) / n for n in L]
    return np.array(list(itertools.product(*axes)))


def plane_wave(L, p, Nv: int, Ns: int, Nc: int, chi: np.ndarray) -> np.ndarray:
    """psi(x) = exp(i p.x) chi, canonical shape; chi has shape (Nv, Ns, Nc) or (Nv, Nc)."""
    Nx, Ny, Nz, Nt = L
    t, z, y, x = np.meshgrid(np.arange(Nt), np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[..., None, None, None] * chi if Ns > 1 else ph[..., None, None] * chi
