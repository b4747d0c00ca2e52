"""The persistent kernel's one-exchange form (pcg_kernel = 2) rearranges the PCG
recurrences as in the CG of Chronopoulos and Gear: u = M^-1 r, w = A u, s = A p carried
by s = w + beta s, gamma = r^T u, delta = u^T A u, beta = gamma / gamma_prev,
alpha = gamma / (delta - beta gamma / alpha_prev).  In exact arithmetic it produces the
iterates of the textbook PCGNR.  This checks that in FP64, on the CPU, against the
oracle's PCGNR on a real linearisation (no GPU): same iterates, same iteration count,
and the stop rule on the recurrence's residual.  It is a statement about the
algorithm of that form, written here from its definition; the CUDA kernel is held to
the oracle by the GPU parity tests."""
import numpy as np

from oracle import ba_oracle as O
from paper_2605_30583_gb300 import synth


def _one_exchange_pcg(J, D, mu, b, precond, tol, max_iters):
    """CG with one inner-product exchange per iteration (Chronopoulos and Gear)."""
    A = lambda v: J.T @ (J @ v) + mu * D * v
    h = np.zeros_like(b)
    r = b.copy()
    u = precond(r)
    p = np.zeros_like(b)
    s = np.zeros_like(b)
    r0 = float(np.sqrt(r @ r))
    gamma_prev = alpha_prev = None
    k = 0
    while k < max_iters:
        w = A(u)                                    # the operator
        gamma, delta, rr = float(r @ u), float(u @ w), float(r @ r)   # the one exchange
        if k > 0 and np.sqrt(rr) <= tol * r0:
            break
        if k == 0:
            beta, alpha = 0.0, gamma / delta
        else:
            beta = gamma / gamma_prev
            alpha = gamma / (delta - beta * gamma / alpha_prev)
        p = u + beta * p
        s = w + beta * s
        h = h + alpha * p
        r = r - alpha * s
        u = precond(r)
        gamma_prev, alpha_prev = gamma, alpha
        k += 1
    return h, k, float(np.sqrt(r @ r))


def _system(seed=31):
    p = synth.make_config("tiny", seed=seed)
    lin = O.linearize(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels)
    D = O.damping_diag(lin.J)
    return lin, D


def test_one_exchange_recurrences_give_the_pcgnr_iterates():
    lin, D = _system()
    mu = 0.01
    pre = O._ba_precond(lin, D, mu)
    for iters in (1, 2, 5, 20):
        ref = O.pcgnr(lin.J, D, mu, -lin.g, pre, tol=0.0, max_iters=iters)
        h, k, _ = _one_exchange_pcg(lin.J, D, mu, -lin.g, pre, tol=0.0, max_iters=iters)
        assert k == ref.iters == iters
        assert np.linalg.norm(h - ref.h) <= 1e-9 * np.linalg.norm(ref.h), iters


def test_one_exchange_stop_rule_matches_pcgnr():
    lin, D = _system(37)
    for mu in (1e-3, 0.1):
        pre = O._ba_precond(lin, D, mu)
        ref = O.pcgnr(lin.J, D, mu, -lin.g, pre, tol=1e-3, max_iters=200)
        h, k, rn = _one_exchange_pcg(lin.J, D, mu, -lin.g, pre, tol=1e-3, max_iters=200)
        assert abs(k - ref.iters) <= 1, (k, ref.iters)
        assert np.linalg.norm(h - ref.h) <= 1e-6 * np.linalg.norm(ref.h)
        # the solution solves the damped system to the tolerance
        res = O.normal_matvec(lin, D, mu, h) + lin.g
        assert np.linalg.norm(res) <= 1.1e-3 * np.linalg.norm(lin.g)


def _one_exchange_pcg_rr(J, D, mu, b, precond, tol, max_iters, drift_at=None, replace=True, max_checks=4):
    """The one-exchange recurrences with residual replacement as the persistent kernel
    runs them: when the recursive residual meets the tolerance, r = b - A h replaces it
    (and u = M^-1 r; p and s are kept) and the solve goes on until a just-replaced (true)
    residual meets it, with at most `max_checks` checks.  `drift_at` plants a drift of
    the recursive residual (scaled by 1e-3 after that update) to show what the checks
    catch."""
    A = lambda v: J.T @ (J @ v) + mu * D * v
    h = np.zeros_like(b)
    r = b.copy()
    u = precond(r)
    p = np.zeros_like(b)
    s = np.zeros_like(b)
    r0 = float(np.sqrt(r @ r))
    gamma_prev = alpha_prev = None
    k = checks = 0
    true_r = False
    while k < max_iters:
        w = A(u)
        gamma, delta, rr = float(r @ u), float(u @ w), float(r @ r)
        if k > 0 and np.sqrt(rr) <= tol * r0:
            if not replace or true_r or checks >= max_checks:
                break
            checks += 1
            r = b - A(h)
            u = precond(r)
            true_r = True
            continue
        if k == 0:
            beta, alpha = 0.0, gamma / delta
        else:
            beta = gamma / gamma_prev
            alpha = gamma / (delta - beta * gamma / alpha_prev)
        p = u + beta * p
        s = w + beta * s
        h = h + alpha * p
        r = r - alpha * s
        if drift_at is not None and k == drift_at:
            r = 1e-3 * r   # the recursive residual drifts away from b - A h
        u = precond(r)
        gamma_prev, alpha_prev = gamma, alpha
        true_r = False
        k += 1
    true_res = float(np.linalg.norm(b - A(h)) / r0)
    return h, k, checks, true_res


def test_residual_replacement_stops_on_a_true_residual():
    lin, D = _system(41)
    mu, tol = 0.01, 1e-3
    pre = O._ba_precond(lin, D, mu)
    b = -lin.g
    # no drift: the checks confirm the recursive residual; the iterates are PCGNR's
    ref = O.pcgnr(lin.J, D, mu, b, pre, tol=tol, max_iters=200)
    h, k, checks, res = _one_exchange_pcg_rr(lin.J, D, mu, b, pre, tol, 200)
    assert checks == 1 and abs(k - ref.iters) <= 1 and res <= tol
    assert np.linalg.norm(h - ref.h) <= 1e-6 * np.linalg.norm(ref.h)
    # a drifted recursive residual: without replacement the solve stops far short of the
    # tolerance; with it, it goes on from the true residual and meets the tolerance
    _, k_plain, _, res_plain = _one_exchange_pcg_rr(lin.J, D, mu, b, pre, tol, 200, drift_at=2, replace=False)
    _, k_rr, checks_rr, res_rr = _one_exchange_pcg_rr(lin.J, D, mu, b, pre, tol, 200, drift_at=2)
    assert res_plain > 10 * tol and k_plain <= 4
    assert res_rr <= tol and k_rr > k_plain and checks_rr >= 1
