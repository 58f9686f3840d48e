"""Local functions written as source text (test inputs, not library code).

The same text is compiled by the library for the GPU and by the oracle for the
host (FP64).  The builtins' bodies are spelled with the same operations in the
same order as the library's builtin functors, so that GPU results can be
compared bitwise with the builtins; GRAY_SCOTT has no builtin counterpart.
"""

JACOBI5 = """
const C u = U(0, 0, 0);
out[0] = fma_(P[0], fma_(C(-4), u, add(add(U(0, -1, 0), U(0, 1, 0)),
                                        add(U(0, 0, -1), U(0, 0, 1)))), u);
"""

DIFF7 = """
const C u = U(0, 0, 0, 0);
const C nb = add(add(add(U(0, -1, 0, 0), U(0, 1, 0, 0)), add(U(0, 0, -1, 0), U(0, 0, 1, 0))),
                 add(U(0, 0, 0, -1), U(0, 0, 0, 1)));
out[0] = fma_(P[0], fma_(C(-6), u, nb), u);
"""

# P = (dt, g, f, H); eta, u, v on a C-grid (see the builtin swe_flux)
SWE_FLUX = """
const C half = C(0.5f), quarter = C(0.25f), mhalf = C(-0.5f);
const C h = P[3], mh = -P[3];
const C e = U(0, 0, 0), eE = U(0, 1, 0), eW = U(0, -1, 0), eN = U(0, 0, 1), eS = U(0, 0, -1);
const C u = U(1, 0, 0), uW = U(1, -1, 0), uE = U(1, 1, 0), uN = U(1, 0, 1), uS = U(1, 0, -1);
const C uWN = U(1, -1, 1);
const C v = U(2, 0, 0), vS = U(2, 0, -1), vN = U(2, 0, 1), vE = U(2, 1, 0), vW = U(2, -1, 0);
const C vES = U(2, 1, -1);
const C dF = fma_(fma_(half, add(e, eE), h), u, mul(fma_(mhalf, add(eW, e), mh), uW));
const C dG = fma_(fma_(half, add(e, eN), h), v, mul(fma_(mhalf, add(eS, e), mh), vS));
out[0] = fma_(-P[0], add(dF, dG), e);
const C vbar = mul(quarter, add(add(v, vE), add(vS, vES)));
const C ubar = mul(quarter, add(add(u, uW), add(uN, uWN)));
const C au = mul(mhalf, fma_(u, sub(uE, uW), mul(vbar, sub(uN, uS))));
const C tu = fma_(P[2], vbar, fma_(-P[1], sub(eE, e), au));
out[1] = fma_(P[0], tu, u);
const C av = mul(mhalf, fma_(ubar, sub(vE, vW), mul(v, sub(vN, vS))));
const C tv = fma_(-P[2], ubar, fma_(-P[1], sub(eN, e), av));
out[2] = fma_(P[0], tv, v);
"""

# Gray-Scott reaction-diffusion, two coupled nonlinear fields (u, v):
#   u' = u + dt (Du L u - u v^2 + F (1 - u)),  v' = v + dt (Dv L v + u v^2 - (F + k) v)
# P = (dt, Du, Dv, F, k); L the 5-point Laplacian.
GRAY_SCOTT = """
const C u = U(0, 0, 0), v = U(1, 0, 0);
const C lu = fma_(C(-4), u, add(add(U(0, -1, 0), U(0, 1, 0)), add(U(0, 0, -1), U(0, 0, 1))));
const C lv = fma_(C(-4), v, add(add(U(1, -1, 0), U(1, 1, 0)), add(U(1, 0, -1), U(1, 0, 1))));
const C uvv = mul(u, mul(v, v));
out[0] = fma_(P[0], fma_(P[1], lu, fma_(P[3], sub(C(1), u), -uvv)), u);
out[1] = fma_(P[0], fma_(P[2], lv, fma_(-add(P[3], P[4]), v, uvv)), v);
"""
GRAY_SCOTT_PRM = [1.0, 0.16, 0.08, 0.035, 0.065]

# Asymmetric taps of radius 2 in 3D (P = (a, b)); products that feed a sum are
# written as fma_, so that the paired FP32 tiles round as the scalar kernels do.
STAR_R2_3D = """
const C u = U(0, 0, 0, 0);
const C far = add(add(U(0, 2, 0, 0), U(0, -2, 0, 0)), add(U(0, 0, 2, 0), U(0, 0, 0, -2)));
const C near = add(add(U(0, 1, 0, 0), U(0, 0, -1, 0)), U(0, 0, 0, 1));
out[0] = fma_(P[0], fma_(C(-4), u, far), fma_(P[1], fma_(C(-3), u, near), u));
"""
