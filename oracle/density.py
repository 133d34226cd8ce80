"""Target weights and the weighted reduced density matrix (oracle; test infrastructure).

Eq. rdensitymatrix (Sec. II.B): rho^L_{alpha,alpha'} = sum_beta sum_l w_l
Phi(l)_{alpha,beta} conj(Phi(l)_{alpha',beta}) over the targeted states; in
sector blocks rho_L(q) = sum_l w_l Psi_l(q) Psi_l(q)^dag, where Psi_l(q) is the
dL(q) x dR(Q_l - q) block of target l in its own sector Q_l.  The printed
dagger placement gives the transpose (= complex conjugate) of this Hermitian
matrix, with the same spectrum.  Each target is normalised first, so that
Tr rho_L = sum_l w_l = 1.

Weights (Sec. II.C): with n targeted states including the ground state, the
ground state and the first and last time targets get 2 Omega, the others
Omega, and 2 Omega * 3 + Omega (n - 3) = 1 gives Omega = 1 / (n + 3).
"""
import numpy as np


def tst_weights(n_v):
    """(w_ground_state, [w_x for the n_v time targets])."""
    if n_v < 2:
        raise ValueError("time-step targeting needs n_v >= 2 (t_0 = 0 < t_{n_v-1} = tau)")
    n = n_v + 1
    omega = 1.0 / (n + 3)
    w = [omega] * n_v
    w[0] = w[-1] = 2 * omega
    return 2 * omega, w


def rho_left(sb, states, weights, real_basis=False):
    """rho_L per left sector (list indexed by left sector, dL x dL complex), states = [(Q, psi)].

    real_basis: the real and imaginary parts of every target are targeted apart with its weight,
    rho_L = sum_l w_l (Re X_l Re X_l^T + Im X_l Im X_l^T) / <psi_l|psi_l> (real symmetric)."""
    rho = [np.zeros((d, d), dtype=complex) for d in sb.ldim]
    for (Q, psi), w in zip(states, weights):
        nrm2 = np.vdot(psi, psi).real
        for qi, ri, off, dl, dr in sb.pairs(Q):
            X = psi[off: off + dl * dr].reshape(dl, dr)
            if real_basis:
                rho[qi] += (w / nrm2) * (X.real @ X.real.T + X.imag @ X.imag.T)
            else:
                rho[qi] += (w / nrm2) * (X @ X.conj().T)
    return rho


def rho_right(sb, states, weights, real_basis=False):
    """rho_R per right sector (the block truncated when a sweep moves left): rho_R[b, b'] =
    sum_l w_l sum_a Psi_l[a, b] conj(Psi_l[a, b']) / <psi_l|psi_l>; real_basis as in rho_left."""
    rho = [np.zeros((d, d), dtype=complex) for d in sb.rdim]
    for (Q, psi), w in zip(states, weights):
        nrm2 = np.vdot(psi, psi).real
        for qi, ri, off, dl, dr in sb.pairs(Q):
            X = psi[off: off + dl * dr].reshape(dl, dr)
            if real_basis:
                rho[ri] += (w / nrm2) * (X.real.T @ X.real + X.imag.T @ X.imag)
            else:
                rho[ri] += (w / nrm2) * (X.T @ X.conj())
    return rho


def rho_eig(rho):
    """Eigenpairs per sector, eigenvalues descending; columns of U are eigenvectors."""
    out = []
    for r in rho:
        lam, U = np.linalg.eigh(r)
        order = np.argsort(-lam, kind="stable")
        out.append((lam[order], U[:, order]))
    return out
