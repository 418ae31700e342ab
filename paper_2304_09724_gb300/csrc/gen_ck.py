"""Writes ck_generated.cuh: straight-line CUDA for the Cauchy-Kovalevskaya (Lax-Wendroff)
procedure of Eq. (2.6) and Section 3.1, for 1D/2D Burgers and 1D/2D Euler.

Method.  At an interface quadrature point the solution is a truncated power series in
(X, Y, t), X = (x - x_p)/dx and Y = (y - y_p)/dy, with normalised coefficients
a[m][n][k] = d^{m+n+k}W/(dX^m dY^n dt^k) / (m! n! k!), m + n + k <= 4.  The spatial slice k = 0
comes in (the upwinded reconstruction); the PDE W_t = -F(W)_x - G(W)_y gives slice k+1 from the
flux series at slice k:
    a[m][n][k+1] = -((m+1)/dx F[m+1][n][k] + (n+1)/dy G[m][n+1][k]) / (k+1).
The flux series come from Cauchy products and quotients of the state series (Euler: u = m/rho,
v = n/rho, mu = m u, mv = m v, nv = n v, p = (g-1)(E - (mu+nv)/2), H = E + p, uH, vH).
The generator walks the dependencies backwards from the outputs a[0][0][k], k = 1..4, and emits
each needed coefficient once, so nothing outside the triangle the outputs depend on is computed.
Run:  python gen_ck.py   (output is committed).
"""
import os


class Gen:
    def __init__(self, dim, eq):
        self.dim, self.eq = dim, eq
        self.lines = []
        self.done = {}
        self.ncomp = 1 if eq == "burgers" else (3 if dim == 1 else 4)
        self.flops = 0

    def idx_ok(self, m, n, k):
        return m >= 0 and n >= 0 and k >= 0 and m + n + k <= 4 and (self.dim == 2 or n == 0)

    def var(self, name, m, n, k):
        """C expression for coefficient (m,n,k) of series `name`; emits code on first use."""
        if not self.idx_ok(m, n, k):
            return None
        key = (name, m, n, k)
        if key in self.done:
            return self.done[key]
        expr = self.build(name, m, n, k)
        if expr is None:
            self.done[key] = None
            return None
        v = f"{name}_{m}{n}{k}"
        self.lines.append(f"  const double {v} = {expr};")
        self.done[key] = v
        return v

    # ---- series definitions ----
    def state_names(self):
        if self.eq == "burgers":
            return ["w0"]
        return ["w0", "w1", "w2"] if self.dim == 1 else ["w0", "w1", "w2", "w3"]

    def build(self, name, m, n, k):
        W = self.state_names()
        if name in W:
            q = W.index(name)
            if k == 0:
                return f"a[{q}][{m * 5 + n}]"
            F = self.var(f"F{q}", m + 1, n, k - 1)
            G = self.var(f"G{q}", m, n + 1, k - 1) if self.dim == 2 else None
            terms = []
            if F is not None:
                terms.append(f"cx[{m}][{k - 1}] * {F}")
            if G is not None:
                terms.append(f"cy[{n}][{k - 1}] * {G}")
            if not terms:
                return None
            self.flops += 2 * len(terms)
            return "-(" + " + ".join(terms) + ")"
        if self.eq == "burgers":
            if name == "uu":
                return self.product("w0", "w0", m, n, k)
            if name in ("F0", "G0"):
                if name == "G0" and self.dim == 1:
                    return None
                uu = self.var("uu", m, n, k)
                if uu is None:
                    return None
                self.flops += 1
                return f"0.5 * {uu}"
            raise KeyError(name)
        # Euler
        if self.dim == 1:
            r, mx, E = W
            if name == "u":
                return self.quotient(mx, r, "u", m, n, k)
            if name == "mu":
                return self.product(mx, "u", m, n, k)
            if name == "p":
                e = self.var(E, m, n, k)
                mu = self.var("mu", m, n, k)
                self.flops += 2
                return f"gm1 * ({e} - 0.5 * {mu})"
            if name == "H":
                self.flops += 1
                return f"{self.var(E, m, n, k)} + {self.var('p', m, n, k)}"
            if name == "uH":
                return self.product("u", "H", m, n, k)
            if name == "F0":
                return self.var(mx, m, n, k)
            if name == "F1":
                self.flops += 1
                return f"{self.var('mu', m, n, k)} + {self.var('p', m, n, k)}"
            if name == "F2":
                return self.var("uH", m, n, k)
            raise KeyError(name)
        r, mx, my, E = W
        if name == "u":
            return self.quotient(mx, r, "u", m, n, k)
        if name == "v":
            return self.quotient(my, r, "v", m, n, k)
        if name == "mu":
            return self.product(mx, "u", m, n, k)
        if name == "mv":
            return self.product(mx, "v", m, n, k)
        if name == "nv":
            return self.product(my, "v", m, n, k)
        if name == "p":
            self.flops += 3
            return f"gm1 * ({self.var(E, m, n, k)} - 0.5 * ({self.var('mu', m, n, k)} + {self.var('nv', m, n, k)}))"
        if name == "H":
            self.flops += 1
            return f"{self.var(E, m, n, k)} + {self.var('p', m, n, k)}"
        if name == "uH":
            return self.product("u", "H", m, n, k)
        if name == "vH":
            return self.product("v", "H", m, n, k)
        if name == "F0":
            return self.var(mx, m, n, k)
        if name == "F1":
            self.flops += 1
            return f"{self.var('mu', m, n, k)} + {self.var('p', m, n, k)}"
        if name == "F2":
            return self.var("mv", m, n, k)
        if name == "F3":
            return self.var("uH", m, n, k)
        if name == "G0":
            return self.var(my, m, n, k)
        if name == "G1":
            return self.var("mv", m, n, k)
        if name == "G2":
            self.flops += 1
            return f"{self.var('nv', m, n, k)} + {self.var('p', m, n, k)}"
        if name == "G3":
            return self.var("vH", m, n, k)
        raise KeyError(name)

    def sub_indices(self, m, n, k):
        for p in range(m + 1):
            for q in range(n + 1):
                for t in range(k + 1):
                    yield p, q, t

    def product(self, A, B, m, n, k):
        terms = []
        for p, q, t in self.sub_indices(m, n, k):
            a = self.var(A, p, q, t)
            b = self.var(B, m - p, n - q, k - t)
            if a is not None and b is not None:
                terms.append(f"{a} * {b}")
        if not terms:
            return None
        self.flops += 2 * len(terms) - 1
        return " + ".join(terms)

    def quotient(self, A, B, name, m, n, k):
        """name = A / B; name[g] = (A[g] - sum_{0 < b <= g} B[b] name[g - b]) / B[0], the sum
        subtracted term by term."""
        a = self.var(A, m, n, k)
        terms = []
        for p, q, t in self.sub_indices(m, n, k):
            if (p, q, t) == (0, 0, 0):
                continue
            b = self.var(B, p, q, t)
            c = self.var(name, m - p, n - q, k - t)
            if b is not None and c is not None:
                terms.append(f"{b} * {c}")
        num = a if a is not None else "0.0"
        if terms:
            # a - t1 - t2 - ... left to right: every step contracts to one fused multiply-add
            num = "(" + num + "".join(f" - {t}" for t in terms) + ")"
            self.flops += 2 * len(terms)
        self.flops += 1
        return f"{num} * inv_r0"

    def emit(self, fname):
        W = self.state_names()
        outs = []
        for q in range(self.ncomp):
            for k in range(1, 5):
                v = self.var(W[q], 0, 0, k)
                outs.append(f"  tc[{q}][{k}] = {v if v is not None else '0.0'};")
        nc = self.ncomp
        head = [
            f"// {fname}: {self.dim}D {self.eq}; inputs a[q][m*5+n] = spatial Taylor coefficients in cell",
            "// units (X = x/dx, Y = y/dy); outputs tc[q][k] = d^k W_q/dt^k / k! for k = 1..4",
            "// (tc[q][0] is left to the caller).  cx[m][k] = (m+1)/((k+1) dx), cy[n][k] = (n+1)/((k+1) dy).",
            f"// FP64 operations (mul/add counted separately): {self.flops}",
            "__device__ __forceinline__ void "
            + f"{fname}(const double (&a)[{nc}][25], double (&tc)[{nc}][5], const double (&cx)[5][4],"
            + " const double (&cy)[5][4], double gm1) {",
            "  (void)gm1; (void)cy;",
        ]
        if self.eq == "euler":
            head.append("  const double inv_r0 = 1.0 / a[0][0];")
        return "\n".join(head + self.lines + outs + ["}"])


def main():
    parts = ["// Generated by gen_ck.py -- do not edit.  Cauchy-Kovalevskaya procedure, Eq. (2.6) and",
             "// Section 3.1, as truncated power-series recursions (see gen_ck.py for the method).",
             "#pragma once", ""]
    stats = []
    for dim, eq, fname in ((1, "burgers", "ck_burgers1d"), (2, "burgers", "ck_burgers2d"),
                           (1, "euler", "ck_euler1d"), (2, "euler", "ck_euler2d")):
        g = Gen(dim, eq)
        parts.append(g.emit(fname))
        parts.append("")
        stats.append((fname, g.flops, len(g.lines)))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ck_generated.cuh")
    with open(out, "w") as f:
        f.write("\n".join(parts))
    for s in stats:
        print("%-14s flops=%5d statements=%4d" % s)


if __name__ == "__main__":
    main()
