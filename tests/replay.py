"""Exact-arithmetic replays of BiCG and GPBiCG (Fig. 5) on tiny systems.

Independent of the oracle's C code: every operation is a rational operation
rounded by tests/exact.py's round-to-nearest-even.  The op order is the one
both implementations follow (each printed product and sum rounded, left to
right), and dot products are exact sums rounded once.
"""
from fractions import Fraction

import exact


def _dot(x, y, p):
    return exact.exact_sum([a.q * b.q for a, b in zip(x, y)], p)


def _spmv(rows, x, p, mode):
    out = []
    for entries in rows:  # entries: list of (col, Val) in column order
        if mode == 0:
            y = exact.Val(Fraction(0))
            for c, a in entries:
                if a.q == 0 or x[c].q == 0:
                    continue
                y = exact.radd(y, exact.rmul(a, x[c], p), p)
        else:
            y = exact.exact_sum([a.q * x[c].q for c, a in entries], p)
        out.append(y)
    return out


def _threshold(rr0, rtol, atol, p):
    rt = exact.Val(Fraction(rtol))
    at = exact.Val(Fraction(atol))
    T = exact.rmul(rt, rt, p)
    A = exact.rmul(at, at, p)
    return exact.radd(exact.rmul(T, rr0, p), A, p)


def _residual(rows, b, x, p):
    return [exact.exact_sum([b[i].q] + [-a.q * x[c].q for c, a in rows[i]], p)
            for i in range(len(b))]


def gpbicg(rows, b, x, p, mode, rtol, maxit):
    """Returns (x, iterations, status, [(r_i, r_i)])."""
    R = exact.rmul
    A_ = exact.radd
    S_ = exact.rsub
    D = exact.rdiv
    n = len(b)
    Z = exact.Val(Fraction(0))
    r = _residual(rows, b, x, p)
    rt = list(r)
    rr0 = _dot(r, r, p)
    thr = _threshold(rr0, rtol, 0.0, p)
    hist = []
    if rr0.q <= thr.q:
        return x, 0, "ok", hist
    rho = _dot(rt, r, p)
    u = [Z] * n
    z = [Z] * n
    s = [Z] * n
    pv = q = t = v = w = y = None
    beta = eta = Z
    zeta = alpha = rho_prev = None
    for i in range(1, maxit + 1):
        if rho.q == 0:
            return x, i - 1, "breakdown", hist
        if i == 1:
            pv = list(r)
            q = _spmv(rows, pv, p, mode)
            d = _dot(rt, q, p)
            alpha = D(rho, d, p)
            aq = [R(alpha, qk, p) for qk in q]
            t = [S_(rk, a, p) for rk, a in zip(r, aq)]
            y = [S_(a, rk, p) for rk, a in zip(r, aq)]
            v = _spmv(rows, t, p, mode)
            mu5 = _dot(v, v, p)
            zeta = D(_dot(v, t, p), mu5, p) if mu5.q != 0 else Z
            eta = Z
        else:
            beta = R(D(rho, rho_prev, p), D(alpha, zeta, p), p)
            w = [A_(vk, R(beta, qk, p), p) for vk, qk in zip(v, q)]
            pv = [A_(rk, R(beta, S_(pk, uk, p), p), p) for rk, pk, uk in zip(r, pv, u)]
            q = _spmv(rows, pv, p, mode)
            alpha = D(rho, _dot(rt, q, p), p)
            s = [S_(tk, rk, p) for tk, rk in zip(t, r)]
            t = [S_(rk, R(alpha, qk, p), p) for rk, qk in zip(r, q)]
            v = _spmv(rows, t, p, mode)
            y = [S_(sk, R(alpha, S_(wk, qk, p), p), p) for sk, wk, qk in zip(s, w, q)]
            mu1, mu2, mu3 = _dot(y, y, p), _dot(v, t, p), _dot(y, t, p)
            mu4, mu5 = _dot(v, y, p), _dot(v, v, p)
            tau = S_(R(mu5, mu1, p), R(mu4, mu4, p), p)
            if tau.q == 0:
                zeta = eta = Z
            else:
                zeta = D(S_(R(mu1, mu2, p), R(mu3, mu4, p), p), tau, p)
                eta = D(S_(R(mu5, mu3, p), R(mu4, mu2, p), p), tau, p)
        u = [A_(R(zeta, qk, p), R(eta, A_(sk, R(beta, uk, p), p), p), p)
             for qk, sk, uk in zip(q, s, u)]
        z = [S_(A_(R(zeta, rk, p), R(eta, zk, p), p), R(alpha, uk, p), p)
             for rk, zk, uk in zip(r, z, u)]
        x = [A_(A_(xk, R(alpha, pk, p), p), zk, p) for xk, pk, zk in zip(x, pv, z)]
        r = [S_(S_(tk, R(eta, yk, p), p), R(zeta, vk, p), p) for tk, yk, vk in zip(t, y, v)]
        rr = _dot(r, r, p)
        hist.append(rr)
        rho_prev, rho = rho, _dot(rt, r, p)
        if rr.q <= thr.q:
            return x, i, "ok", hist
        if zeta.q == 0:
            return x, i, "breakdown", hist
    return x, maxit, "noconv", hist


def bicg(rows, rows_t, b, x, p, mode, rtol, maxit):
    R = exact.rmul
    A_ = exact.radd
    S_ = exact.rsub
    D = exact.rdiv
    r = _residual(rows, b, x, p)
    rt = list(r)
    rr0 = _dot(r, r, p)
    thr = _threshold(rr0, rtol, 0.0, p)
    hist = []
    if rr0.q <= thr.q:
        return x, 0, "ok", hist
    rho = _dot(rt, r, p)
    pv = pt = rho_prev = None
    for i in range(1, maxit + 1):
        if rho.q == 0:
            return x, i - 1, "breakdown", hist
        if i == 1:
            pv, pt = list(r), list(rt)
        else:
            beta = D(rho, rho_prev, p)
            pv = [A_(rk, R(beta, pk, p), p) for rk, pk in zip(r, pv)]
            pt = [A_(rk, R(beta, pk, p), p) for rk, pk in zip(rt, pt)]
        z = _spmv(rows, pv, p, mode)
        zt = _spmv(rows_t, pt, p, mode)
        alpha = D(rho, _dot(pt, z, p), p)
        x = [A_(xk, R(alpha, pk, p), p) for xk, pk in zip(x, pv)]
        r = [S_(rk, R(alpha, zk, p), p) for rk, zk in zip(r, z)]
        rt = [S_(rk, R(alpha, zk, p), p) for rk, zk in zip(rt, zt)]
        rr = _dot(r, r, p)
        hist.append(rr)
        rho_prev, rho = rho, _dot(rt, r, p)
        if rr.q <= thr.q:
            return x, i, "ok", hist
    return x, maxit, "noconv", hist


def cgs(rows, b, x, p, mode, rtol, maxit):
    """CGS in the textbook order (each product and sum rounded, left to right)."""
    R = exact.rmul
    A_ = exact.radd
    S_ = exact.rsub
    D = exact.rdiv
    r = _residual(rows, b, x, p)
    rt = list(r)
    rr0 = _dot(r, r, p)
    thr = _threshold(rr0, rtol, 0.0, p)
    hist = []
    if rr0.q <= thr.q:
        return x, 0, "ok", hist
    rho = _dot(rt, r, p)
    u = pv = q = rho_prev = None
    for i in range(1, maxit + 1):
        if rho.q == 0:
            return x, i - 1, "breakdown", hist
        if i == 1:
            u, pv = list(r), list(r)
        else:
            beta = D(rho, rho_prev, p)
            u = [A_(rk, R(beta, qk, p), p) for rk, qk in zip(r, q)]
            pv = [A_(uk, R(beta, A_(qk, R(beta, pk, p), p), p), p)
                  for uk, qk, pk in zip(u, q, pv)]
        v = _spmv(rows, pv, p, mode)
        d = _dot(rt, v, p)
        if d.q == 0:
            return x, i - 1, "breakdown", hist
        alpha = D(rho, d, p)
        q = [S_(uk, R(alpha, vk, p), p) for uk, vk in zip(u, v)]
        w = [A_(uk, qk, p) for uk, qk in zip(u, q)]
        x = [A_(xk, R(alpha, wk, p), p) for xk, wk in zip(x, w)]
        aw = _spmv(rows, w, p, mode)
        r = [S_(rk, R(alpha, ak, p), p) for rk, ak in zip(r, aw)]
        rr = _dot(r, r, p)
        hist.append(rr)
        rho_prev, rho = rho, _dot(rt, r, p)
        if rr.q <= thr.q:
            return x, i, "ok", hist
    return x, maxit, "noconv", hist


def bicgstab(rows, b, x, p, mode, rtol, maxit):
    """BiCGSTAB in the textbook order; omega = +0 when (t, t) = 0."""
    R = exact.rmul
    A_ = exact.radd
    S_ = exact.rsub
    D = exact.rdiv
    Z = exact.Val(Fraction(0))
    r = _residual(rows, b, x, p)
    rt = list(r)
    rr0 = _dot(r, r, p)
    thr = _threshold(rr0, rtol, 0.0, p)
    hist = []
    if rr0.q <= thr.q:
        return x, 0, "ok", hist
    rho = _dot(rt, r, p)
    pv = v = rho_prev = None
    alpha = omega = Z
    for i in range(1, maxit + 1):
        if rho.q == 0:
            return x, i - 1, "breakdown", hist
        if i == 1:
            pv = list(r)
        else:
            beta = R(D(rho, rho_prev, p), D(alpha, omega, p), p)
            pv = [A_(rk, R(beta, S_(pk, R(omega, vk, p), p), p), p)
                  for rk, pk, vk in zip(r, pv, v)]
        v = _spmv(rows, pv, p, mode)
        d = _dot(rt, v, p)
        if d.q == 0:
            return x, i - 1, "breakdown", hist
        alpha = D(rho, d, p)
        s = [S_(rk, R(alpha, vk, p), p) for rk, vk in zip(r, v)]
        t = _spmv(rows, s, p, mode)
        tt = _dot(t, t, p)
        omega = D(_dot(t, s, p), tt, p) if tt.q != 0 else Z
        x = [A_(A_(xk, R(alpha, pk, p), p), R(omega, sk, p), p)
             for xk, pk, sk in zip(x, pv, s)]
        r = [S_(sk, R(omega, tk, p), p) for sk, tk in zip(s, t)]
        rr = _dot(r, r, p)
        hist.append(rr)
        rho_prev, rho = rho, _dot(rt, r, p)
        if rr.q <= thr.q:
            return x, i, "ok", hist
        if omega.q == 0:
            return x, i, "breakdown", hist
    return x, maxit, "noconv", hist


def ilu0(rows, p):
    """ILU(0) in the textbook IKJ order; rows: list of [(col, Val)] sorted by
    column.  Returns the factor rows (L left of the diagonal, U from it)."""
    lu = [list(r) for r in rows]
    pos = [{c: k for k, (c, _) in enumerate(r)} for r in lu]
    for i, row in enumerate(lu):
        for a in range(len(row)):
            k = row[a][0]
            if k >= i:
                break
            ukk = lu[k][pos[k][k]][1]
            q = exact.rdiv(row[a][1], ukk, p)
            row[a] = (k, q)
            for b in range(a + 1, len(row)):
                j = row[b][0]
                if j in pos[k]:
                    ukj = lu[k][pos[k][j]][1]
                    row[b] = (j, exact.rsub(row[b][1], exact.rmul(q, ukj, p), p))
    return lu


def ilu0_apply(lu, r, p):
    """w = (LU)^{-1} r: forward over rows, then backward from the last row."""
    n = len(lu)
    w = [None] * n
    for i in range(n):
        acc = r[i]
        for c, v in lu[i]:
            if c >= i:
                break
            acc = exact.rsub(acc, exact.rmul(v, w[c], p), p)
        w[i] = acc
    for i in range(n - 1, -1, -1):
        acc = w[i]
        d = None
        for c, v in lu[i]:
            if c == i:
                d = v
            elif c > i:
                acc = exact.rsub(acc, exact.rmul(v, w[c], p), p)
        w[i] = exact.rdiv(acc, d, p)
    return w


def bicgstab_ilu0(rows, b, x, p, mode, rtol, maxit, side="left"):
    """BiCGSTAB preconditioned with ILU(0) K = LU.  Left (the paper's,
    Section 4.2): BiCGSTAB on K^{-1}A x = K^{-1}b, the residual carried and
    tested is r^ = K^{-1}(b - A x).  Right: p^ = K^{-1} p, s^ = K^{-1} s."""
    if side == "left":
        return _bicgstab_left(rows, b, x, p, mode, rtol, maxit)
    R = exact.rmul
    A_ = exact.radd
    S_ = exact.rsub
    D = exact.rdiv
    Z = exact.Val(Fraction(0))
    lu = ilu0(rows, p)
    r = _residual(rows, b, x, p)
    rt = list(r)
    rr0 = _dot(r, r, p)
    thr = _threshold(rr0, rtol, 0.0, p)
    hist = []
    if rr0.q <= thr.q:
        return x, 0, "ok", hist
    rho = _dot(rt, r, p)
    pv = v = rho_prev = None
    alpha = omega = Z
    for i in range(1, maxit + 1):
        if rho.q == 0:
            return x, i - 1, "breakdown", hist
        if i == 1:
            pv = list(r)
        else:
            beta = R(D(rho, rho_prev, p), D(alpha, omega, p), p)
            pv = [A_(rk, R(beta, S_(pk, R(omega, vk, p), p), p), p)
                  for rk, pk, vk in zip(r, pv, v)]
        ph = ilu0_apply(lu, pv, p)
        v = _spmv(rows, ph, p, mode)
        d = _dot(rt, v, p)
        if d.q == 0:
            return x, i - 1, "breakdown", hist
        alpha = D(rho, d, p)
        s = [S_(rk, R(alpha, vk, p), p) for rk, vk in zip(r, v)]
        sh = ilu0_apply(lu, s, p)
        t = _spmv(rows, sh, p, mode)
        tt = _dot(t, t, p)
        omega = D(_dot(t, s, p), tt, p) if tt.q != 0 else Z
        x = [A_(A_(xk, R(alpha, pk, p), p), R(omega, sk, p), p)
             for xk, pk, sk in zip(x, ph, sh)]
        r = [S_(sk, R(omega, tk, p), p) for sk, tk in zip(s, t)]
        rr = _dot(r, r, p)
        hist.append(rr)
        rho_prev, rho = rho, _dot(rt, r, p)
        if rr.q <= thr.q:
            return x, i, "ok", hist
        if omega.q == 0:
            return x, i, "breakdown", hist
    return x, maxit, "noconv", hist


def _bicgstab_left(rows, b, x, p, mode, rtol, maxit):
    R = exact.rmul
    A_ = exact.radd
    S_ = exact.rsub
    D = exact.rdiv
    Z = exact.Val(Fraction(0))
    lu = ilu0(rows, p)
    r = ilu0_apply(lu, _residual(rows, b, x, p), p)
    rt = list(r)
    rr0 = _dot(r, r, p)
    thr = _threshold(rr0, rtol, 0.0, p)
    hist = []
    if rr0.q <= thr.q:
        return x, 0, "ok", hist
    rho = _dot(rt, r, p)
    pv = v = rho_prev = None
    alpha = omega = Z
    for i in range(1, maxit + 1):
        if rho.q == 0:
            return x, i - 1, "breakdown", hist
        if i == 1:
            pv = list(r)
        else:
            beta = R(D(rho, rho_prev, p), D(alpha, omega, p), p)
            pv = [A_(rk, R(beta, S_(pk, R(omega, vk, p), p), p), p)
                  for rk, pk, vk in zip(r, pv, v)]
        v = ilu0_apply(lu, _spmv(rows, pv, p, mode), p)
        d = _dot(rt, v, p)
        if d.q == 0:
            return x, i - 1, "breakdown", hist
        alpha = D(rho, d, p)
        s = [S_(rk, R(alpha, vk, p), p) for rk, vk in zip(r, v)]
        t = ilu0_apply(lu, _spmv(rows, s, p, mode), p)
        tt = _dot(t, t, p)
        omega = D(_dot(t, s, p), tt, p) if tt.q != 0 else Z
        x = [A_(A_(xk, R(alpha, pk, p), p), R(omega, sk, p), p)
             for xk, pk, sk in zip(x, pv, s)]
        r = [S_(sk, R(omega, tk, p), p) for sk, tk in zip(s, t)]
        rr = _dot(r, r, p)
        hist.append(rr)
        rho_prev, rho = rho, _dot(rt, r, p)
        if rr.q <= thr.q:
            return x, i, "ok", hist
        if omega.q == 0:
            return x, i, "breakdown", hist
    return x, maxit, "noconv", hist
