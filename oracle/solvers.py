"""Solvers of the oracle (test infrastructure).

* ``cg``: textbook conjugate gradient for a Hermitian positive-definite operator
  (Sec. 2.1, "we invert using ... conjugate gradient"; Table 3.1), zero initial guess,
  stopped on the true relative residual ||b - A x|| / ||b||.
* ``shifted_solve``: x_i = (J - z_i)^{-1} b for complex shifts z_i (App. C, eq.
  force_polycorr).  The paper's multi-shift CG reaches these from one Krylov space; the
  oracle takes the plain definition instead and solves each shifted system on its own,
  by CG on the normal equations (J - z)^dag (J - z) x = (J - z)^dag b, all shifts as one
  batch.  J Hermitian makes (J - z)^dag = J - conj(z).
* ``dense_solve``: brute force with LU on an assembled matrix.

Vectors carry an optional leading batch dimension; inner products are taken per batch
entry over all remaining dimensions.
"""
import torch


def _dot(a, b):
    """<a, b> = sum conj(a) b per leading batch entry (shape (B,) or scalar)."""
    return (a.conj() * b).reshape(a.shape[0], -1).sum(-1) if a.dim() > 6 else (a.conj() * b).sum()


def _bcast(s, v):
    return s.reshape(s.shape + (1,) * (v.dim() - s.dim()))


def cg(A, b, tol=1e-12, maxiter=10000):
    """Solve A x = b for HPD A; returns (x, iterations, true relative residual)."""
    x = torch.zeros_like(b)
    r = b.clone()
    p = r.clone()
    rr = _dot(r, r).real
    bb = rr.clone()
    it = 0
    while it < maxiter:
        if bool(torch.all(torch.sqrt(rr / bb) < tol)):
            break
        Ap = A(p)
        live = torch.sqrt(rr / bb) >= tol
        alpha = torch.where(live, rr / _dot(p, Ap).real, torch.zeros_like(rr))
        x = x + _bcast(alpha, x) * p
        r = r - _bcast(alpha, r) * Ap
        rr_new = _dot(r, r).real
        beta = torch.where(live, rr_new / rr, torch.zeros_like(rr))
        p = torch.where(_bcast(live, p), r + _bcast(beta, p) * p, p)
        rr = torch.where(live, rr_new, rr)
        it += 1
    res = torch.sqrt(_dot(b - A(x), b - A(x)).real / bb)
    return x, it, res


def shifted_solve(J, b, shifts, tol=1e-12, maxiter=10000):
    """x[i] = (J - z_i)^{-1} b for each complex z_i, by batched CG on the normal equations.

    ``b`` has no batch dimension; the result has a leading dimension len(shifts)."""
    z = torch.as_tensor(shifts, dtype=torch.complex128)
    nb = z.numel()
    B = b.unsqueeze(0).expand(nb, *b.shape).clone()

    def op(v):
        return J(v) - _bcast(z, v) * v

    def op_dag(v):
        return J(v) - _bcast(z.conj(), v) * v

    def normal(v):
        return op_dag(op(v))

    rhs = op_dag(B)
    x, it, _ = cg(normal, rhs, tol=tol * 1e-1, maxiter=maxiter)
    res = torch.sqrt(_dot(B - op(x), B - op(x)).real / _dot(B, B).real)
    return x, it, res


def dense_solve(Mat, b):
    return torch.linalg.solve(Mat, b)


def multishift_cg(A, b, sigmas, tol=1e-12, maxiter=10000):
    """x_s = (A + sigma_s)^{-1} b for all complex shifts from the Krylov space of the HPD
    seed A, by the shifted CG recurrences (the multi-shift CG the paper uses for the
    poly-correction term, Sec. 3.1 and App. C; Jegerlehner, hep-lat/9612014).

    The shifted residuals stay collinear with the seed residual, r_s = zeta_s r, and
      zeta_s(n+1) = zeta_s(n) zeta_s(n-1) alpha(n-1) /
          [alpha(n-1) zeta_s(n-1) (1 + alpha(n) sigma_s) + alpha(n) beta(n-1) (zeta_s(n-1) - zeta_s(n))]
      alpha_s(n) = alpha(n) zeta_s(n+1) / zeta_s(n),  beta_s(n) = beta(n) (zeta_s(n+1) / zeta_s(n))^2.
    Stops when every shifted residual |zeta_s| ||r|| and the seed residual are below
    tol ||b||.  Returns (x[s, ...], iterations)."""
    sig = torch.as_tensor(sigmas, dtype=torch.complex128)
    ns = sig.numel()
    x = torch.zeros(ns, *b.shape, dtype=b.dtype)
    p = b.unsqueeze(0).expand(ns, *b.shape).clone()
    r = b.clone()
    pr = b.clone()                       # seed search direction
    rr = _dot(r, r).real
    bb = rr.clone()
    zeta_prev = torch.ones(ns, dtype=torch.complex128)
    zeta = torch.ones(ns, dtype=torch.complex128)
    alpha_prev, beta_prev = 1.0, 0.0
    it = 0
    while it < maxiter:
        res = torch.sqrt(rr / bb).item()
        if res < tol and bool(torch.all(zeta.abs() * res < tol)):
            break
        w = A(pr)
        alpha = (rr / _dot(pr, w).real).item()
        zeta_next = zeta * zeta_prev * alpha_prev / (
            alpha_prev * zeta_prev * (1 + alpha * sig) + alpha * beta_prev * (zeta_prev - zeta))
        alpha_s = alpha * zeta_next / zeta
        x = x + _bcast(alpha_s, x) * p
        r = r - alpha * w
        rr_new = _dot(r, r).real
        beta = (rr_new / rr).item()
        beta_s = beta * (zeta_next / zeta) ** 2
        p = _bcast(zeta_next, p) * r.unsqueeze(0) + _bcast(beta_s, p) * p
        pr = r + beta * pr
        zeta_prev, zeta = zeta, zeta_next
        alpha_prev, beta_prev = alpha, beta
        rr = rr_new
        it += 1
    return x, it
