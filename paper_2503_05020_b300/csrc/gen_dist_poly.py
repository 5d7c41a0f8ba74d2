"""Generate dist_poly.cuh: value, gradient and packed upper Hessian of the polynomial pieces of
the squared point-edge, point-triangle and edge-edge distances used by the CUDA contact kernels.

    point-edge:      d^2 = C / D,   C = |(e0 - p) x (e1 - p)|^2,  D = |e1 - e0|^2
    point-triangle:  d^2 = N^2 / D, N = (p - t0) . n,  n = (t1 - t0) x (t2 - t0),  D = |n|^2
    edge-edge:       d^2 = N^2 / D, N = (b0 - a0) . n, n = (a1 - a0) x (b1 - b0),  D = |n|^2

The edge-edge D is also the argument of the parallel-edge mollifier. The quotient rule that
turns these pieces into derivatives of d^2 is written by hand in the kernels. Run:
    python gen_dist_poly.py > dist_poly.cuh
"""
import sympy as sp


def vec(name):
    return sp.Matrix(sp.symbols(f"{name}_0:3", real=True))


def emit(fname, args, pieces):
    """pieces: list of (name, expr, vars) -> value, grad[n], hess packed upper [n(n+1)/2]."""
    outs = []
    names = []
    for name, expr, vs in pieces:
        n = len(vs)
        outs.append(expr)
        names.append(f"{name}_val[0]")
        g = [sp.diff(expr, v) for v in vs]
        for i in range(n):
            outs.append(g[i])
            names.append(f"{name}_grad[{i}]")
        k = 0
        for i in range(n):
            for j in range(i, n):
                outs.append(sp.diff(g[i], vs[j]))
                names.append(f"{name}_hess[{k}]")
                k += 1
    reps, red = sp.cse(outs, optimizations="basic")
    sig = ", ".join(f"const double* __restrict__ {a}" for a in args)
    outsig = ", ".join(f"double* __restrict__ {nm}_val, double* __restrict__ {nm}_grad, double* __restrict__ {nm}_hess"
                       for nm, _, _ in pieces)
    lines = [f"__device__ __forceinline__ void {fname}({sig}, {outsig}) {{"]
    for a in args:
        for i in range(3):
            lines.append(f"  const double {a}_{i} = {a}[{i}];")
    for s, e in reps:
        lines.append(f"  const double {s} = {sp.ccode(e)};")
    for nm, e in zip(names, red):
        lines.append(f"  {nm} = {sp.ccode(e)};")
    lines.append("}")
    return "\n".join(lines)


def main():
    p, e0, e1, t0, t1, t2, a0, a1, b0, b1 = (vec(n) for n in ["p", "e0", "e1", "t0", "t1", "t2", "a0", "a1", "b0", "b1"])
    out = ["// Generated by gen_dist_poly.py (sympy). Do not edit by hand.",
           "// Packed upper Hessians: entry (i, j), i <= j, at i*n - i*(i-1)/2 + (j - i).",
           "#pragma once", ""]
    # point-edge (9 variables: p, e0, e1)
    vs = list(p) + list(e0) + list(e1)
    c = (e0 - p).cross(e1 - p)
    C = c.dot(c)
    D = (e1 - e0).dot(e1 - e0)
    out.append(emit("pe_poly", ["p", "e0", "e1"], [("C", C, vs), ("D", D, vs)]))
    out.append("")
    # point-triangle (12 variables: p, t0, t1, t2)
    vs = list(p) + list(t0) + list(t1) + list(t2)
    n = (t1 - t0).cross(t2 - t0)
    N = (p - t0).dot(n)
    D = n.dot(n)
    out.append(emit("pt_poly", ["p", "t0", "t1", "t2"], [("N", N, vs), ("D", D, vs)]))
    out.append("")
    # edge-edge (12 variables: a0, a1, b0, b1)
    vs = list(a0) + list(a1) + list(b0) + list(b1)
    n = (a1 - a0).cross(b1 - b0)
    N = (b0 - a0).dot(n)
    D = n.dot(n)
    out.append(emit("ee_poly", ["a0", "a1", "b0", "b1"], [("N", N, vs), ("D", D, vs)]))
    print("\n".join(out))


if __name__ == "__main__":
    main()
