"""Lanczos tridiagonalisation started from phi and the Krylov exponential (oracle; test infrastructure).

Sec. II.A: Lanczos run from the state phi itself (not a random vector) gives
V (n_l Lanczos vectors) and the tridiagonal T; T = S^dag D S is diagonalised
(cheap, n_l x n_l); then phi(t) ~ V^dag S^dag e^{-i D t} S V phi.  Because the
recursion starts at phi, V phi = ||phi|| e_0, so
    phi(t) = ||phi|| sum_k v_k [S^dag e^{-i D t} S]_{k,0}.
The printed Eq. lanczosevolution carries extra T factors and e^{+i d t}; the
T factors cannot be right (T is not unitary) and the time sign only conjugates
the result for real H and real phi, so the oracle uses exp(-iHt).
Sec. II.C, Eq. lanczosevolution2: phi(t + tau) is obtained from phi(t) by the
same formula; applied repeatedly it reaches any time.
Sec. II.B: the n_v time targets phi(t + t_x), t_0 = 0 < ... < t_{n_v-1} = tau,
all come from the one Krylov space built at phi(t); t_x = x tau / (n_v - 1).

Lanczos step (full re-orthogonalisation):
    w = H v_j;  alpha_j = Re <v_j|w>;  w -= alpha_j v_j + beta_j v_{j-1};
    two passes of classical Gram-Schmidt against v_0..v_j;  beta_{j+1} = ||w||;
    stop at n_K vectors or at breakdown beta_{j+1} <= tol * max(1, |alpha_j|).
Error estimate (Saad 1992): ||phi|| beta_n |[e^{-i T tau}]_{n-1,0}|.
"""
import numpy as np


def lanczos(apply_h, phi, nk, tol=1e-12):
    """Returns (V list, alpha, beta, beta0, beta_n); beta[j] couples v_j and v_{j+1}."""
    beta0 = np.linalg.norm(phi)
    V = [phi / beta0]
    alpha, beta = [], []
    beta_n = 0.0
    for j in range(nk):
        w = apply_h(V[j])
        a = np.vdot(V[j], w).real
        w = w - a * V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        for _ in range(2):                      # classical Gram-Schmidt, twice
            h = np.array([np.vdot(v, w) for v in V])
            for k, v in enumerate(V):
                w = w - h[k] * v
        b = np.linalg.norm(w)
        alpha.append(a)
        beta_n = b
        if j == nk - 1 or b <= tol * max(1.0, abs(a)):
            break
        beta.append(b)
        V.append(w / b)
    return V, np.array(alpha), np.array(beta), beta0, beta_n


def tridiagonal(alpha, beta):
    n = len(alpha)
    T = np.diag(alpha).astype(float)
    for k in range(n - 1):
        T[k, k + 1] = T[k + 1, k] = beta[k]
    return T


def krylov_coefficients(alpha, beta, beta0, times):
    """c_x[k] = ||phi|| [S^dag e^{-i D t_x} S]_{k,0} for each time t_x (T = S^dag D S)."""
    T = tridiagonal(alpha, beta)
    d, cols = np.linalg.eigh(T)
    S = cols.T                                   # rows of S are the eigenvectors: T = S^T diag(d) S
    out = []
    for t in times:
        out.append(beta0 * (S.conj().T @ (np.exp(-1j * d * t) * S[:, 0])))
    return np.array(out)


def error_estimate(alpha, beta, beta0, beta_n, tau):
    n = len(alpha)
    c = krylov_coefficients(alpha, beta, 1.0, [tau])[0]
    return beta0 * beta_n * abs(c[n - 1])


def target_times(tau, n_v):
    return [x * tau / (n_v - 1) for x in range(n_v)]


def evolve(apply_h, phi, times, nk, tol=1e-12):
    """Targets phi(t_x) for each t_x from one Krylov space at phi; returns (targets, n_used, err_est)."""
    V, alpha, beta, beta0, beta_n = lanczos(apply_h, phi, nk, tol)
    C = krylov_coefficients(alpha, beta, beta0, times)
    targets = [sum(c[k] * V[k] for k in range(len(V))) for c in C]
    return targets, len(alpha), error_estimate(alpha, beta, beta0, beta_n, max(times))


def time_steps(apply_h, phi, tau, n_steps, n_v, nk, tol=1e-12):
    """Repeated advance (Eq. lanczosevolution2): list over steps of the n_v targets."""
    times = target_times(tau, n_v)
    out, cur = [], phi
    for _ in range(n_steps):
        targets, n_used, err = evolve(apply_h, cur, times, nk, tol)
        out.append((targets, n_used, err))
        cur = targets[-1]
    return out
