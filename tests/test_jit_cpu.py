"""Local functions written as source, compiled at run time (no GPU needed).

lope_stencil_create_source wraps the body in a functor with the builtins'
interface and NVRTC compiles it into the library's kernel templates (TMA
tiles / z-march, trapezoid tiles, direct kernel and their Runge-Kutta stage
forms) for sm_103a.  Compilation needs no device, so these tests run on the
CPU: they check that every kernel instance compiles for every storage type and
that a body with an error reports the compiler's message.
"""
import pytest

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

BOX_TWO_FIELDS = """
// a coupled pair with corner taps, written with operators
out[0] = U(0, 0, 0) + P[0] * (U(1, 1, 1) - U(1, -1, -1));
out[1] = U(1, 0, 0) - P[1] * (U(0, 1, -1) - U(0, -1, 1));
"""


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_source_stencils_compile_for_every_storage_type(lope, dtype):
    lope.Stencil.source(JACOBI5, ndim=2, radius=1, params=[0.2]).compile(dtype)
    lope.Stencil.source(DIFF7, ndim=3, radius=1, params=[0.1]).compile(dtype)
    lope.Stencil.source(BOX_TWO_FIELDS, ndim=2, radius=1, nfields=2, params=[0.1, 0.05],
                        box=True).compile(dtype)


def test_radius_two_and_three_fields_compile(lope):
    body = """
for (int f = 0; f < 3; ++f)
  out[f] = fma_(P[f], sub(add(U(f, -2, 0), U(f, 0, 2)), add(U(f, 2, 0), U(f, 0, -2))), U(f, 0, 0));
"""
    lope.Stencil.source(body, ndim=2, radius=2, nfields=3, params=[0.1, 0.2, 0.3]).compile("f32")


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_3d_radius_two_star_and_three_fields_compile(lope, dtype):
    """3D instances beyond diff7: a radius-2 star function (TMA z-march, and for
    FP32 / FP64 the z-march with copied planes) and three coupled fields."""
    star_r2 = """
const C u = U(0, 0, 0, 0);
const C far = add(add(U(0, 2, 0, 0), U(0, -2, 0, 0)), add(U(0, 0, 2, 0), U(0, 0, 0, -2)));
out[0] = fma_(P[0], fma_(C(-4), u, far), u);
"""
    three = """
for (int f = 0; f < 3; ++f)
  out[f] = fma_(P[0], sub(U((f + 1) % 3, 0, 0, 1), U(f, 1, 0, 0)), U(f, 0, 0, 0));
"""
    lope.Stencil.source(star_r2, ndim=3, radius=2, params=[0.05]).compile(dtype)
    lope.Stencil.source(three, ndim=3, radius=1, nfields=3, params=[0.1]).compile(dtype)


def test_compile_error_reports_the_compiler_log(lope):
    st = lope.Stencil.source("out[0] = U(0, 0, 0) + undefined_name;", params=[1.0])
    with pytest.raises(lope.LopeError, match="undefined_name"):
        st.compile("f32")


def test_bad_arguments_are_rejected(lope):
    with pytest.raises(lope.LopeError, match="radius"):
        lope.Stencil.source(JACOBI5, ndim=2, radius=3)
    with pytest.raises(lope.LopeError, match="nfields"):
        lope.Stencil.source(JACOBI5, ndim=2, radius=1, nfields=4)
    with pytest.raises(lope.LopeError, match="8 parameters"):
        lope.Stencil.source(JACOBI5, params=[0.0] * 9)
    with pytest.raises(lope.LopeError, match="non-finite"):
        lope.Stencil.source(JACOBI5, params=[float("nan")])


def test_literal_taps_outside_the_declared_halo_are_refused(lope):
    """Sec. 3.5: a local function may not index outside its halo."""
    with pytest.raises(lope.LopeError, match="beyond the declared halo"):
        lope.Stencil.source("out[0] = U(0, 2, 0);", ndim=2, radius=1)
    with pytest.raises(lope.LopeError, match="beyond the declared halo"):
        lope.Stencil.source("out[0] = U(0, 0, 0, -3);", ndim=3, radius=2)
    with pytest.raises(lope.LopeError, match="corner"):
        lope.Stencil.source("out[0] = U(0, 1, 1);", ndim=2, radius=1)
    with pytest.raises(lope.LopeError, match="field"):
        lope.Stencil.source("out[0] = U(1, 0, 0);", ndim=2, radius=1, nfields=1)
    with pytest.raises(lope.LopeError, match="number of arguments"):
        lope.Stencil.source("out[0] = U(0, 1, 0, 0);", ndim=2, radius=1)
    # within the halo, a declared box function, comments and computed taps pass
    lope.Stencil.source("out[0] = U(0, 1, 1); // U(0, 5, 0) in a comment", ndim=2, radius=1,
                        box=True)
    lope.Stencil.source("C s = C(0);\nfor (int d = -1; d <= 1; ++d) s = add(s, U(0, d, 0));\n"
                        "out[0] = s; /* U(0, 9, 9) */", ndim=2, radius=1)
