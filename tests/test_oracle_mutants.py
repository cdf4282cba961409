"""The oracle's pins catch plausible mistakes.

Each case compiles a copy of the oracle with one planted mistake (a swapped
operand, a wrong sign or index, a dropped negation) and checks that at least
one pin of test_oracle_pins fails against it.  Mistakes are planted only in
the CPU oracle.
"""
import pytest

import oracle
from tests import test_oracle_pins as P

# (name, [(original text, mutated text), ...]); every original must occur once
MUTANTS = [
    ("interpolation weights swapped",
     [("const R vel = (R(1) - s) * ua + s * ub;", "const R vel = s * ua + (R(1) - s) * ub;")]),
    ("gray point interpolated along the wrong edge",
     [("u[(size_t)(m.j + 1) * (nx + 1) + m.i], lam, f);",
       "u[(size_t)m.j * (nx + 1) + m.i + 1], lam, f);")]),
    ("circle coefficient sign",
     [("const double al = r2 * qy - q2 * ry;", "const double al = q2 * ry - r2 * qy;")]),
    ("wrong root of the circle",
     [("if (a_with_T && !b_with_T) yrel = yb;", "if (!a_with_T && b_with_T) yrel = yb;")]),
    ("corner flip off by one",
     [("for (int kk = std::min(i, p.ix) + 1; kk <= std::max(i, p.ix); ++kk) N.k(kk, j) ^= 1;",
       "for (int kk = std::min(i, p.ix); kk < std::max(i, p.ix); ++kk) N.k(kk, j) ^= 1;")]),
    ("aligned marker keeps its old fraction",
     [("land.push_back({p.ix, j, p.fx, i});", "land.push_back({p.ix, j, S.hc(i, j), i});")]),
    ("centre colour not negated",
     [("const int vr = lr < 0 ? -1 : !N.kc(k, lr);", "const int vr = lr < 0 ? -1 : N.kc(k, lr);"),
      ("const int vl = ll < 0 ? -1 : !N.kc(k, ll);", "const int vl = ll < 0 ? -1 : N.kc(k, ll);")]),
    ("triangle leg measured from the wrong corner",
     [("case 1: a = 1.0 - s[0]; b = s[1]; break;", "case 1: a = s[0]; b = s[1]; break;")]),
    ("four-marker fraction inverted",
     [("return zc == 0 ? Tsum : 1.0 - Tsum;", "return zc == 1 ? Tsum : 1.0 - Tsum;")]),
    ("trapezoid side swapped",
     [("return c[0] ? 0.5 * (s[0] + s[2]) : 0.5 * ((1.0 - s[0]) + (1.0 - s[2]));",
       "return c[0] ? 0.5 * ((1.0 - s[0]) + (1.0 - s[2])) : 0.5 * (s[0] + s[2]);")]),
    ("second difference sign",
     [("const R hpp = (h[2] - h[1]) - (h[1] - h[0]);", "const R hpp = (h[2] - h[1]) + (h[1] - h[0]);")]),
    ("height direction swapped",
     [("const bool ycol = ax >= ay;", "const bool ycol = ax < ay;")]),
    ("circle root at initialisation on the wrong side",
     [("const double root = P.in_circle(o, xi, yj) ? sc->xc[o] + sq : sc->xc[o] - sq;",
       "const double root = P.in_circle(o, xi, yj) ? sc->xc[o] - sq : sc->xc[o] + sq;")]),
    ("y sweep maps edges without transposing fractions",
     [("for (int i = 0; i < S.nx; ++i) T.v(j, i) = S.hc(i, j);",
       "for (int i = 0; i < S.nx; ++i) T.v(j, i) = R(1) - S.hc(i, j);")]),
    ("parabola fit: tangent and normal coordinates swapped",
     [("const R sv = ddx * ny - ddy * nx;  // along the tangent (ny, -nx)",
       "const R sv = ddx * nx + ddy * ny;  // along the tangent (ny, -nx)"),
      ("const R zv = ddx * nx + ddy * ny;  // along the normal",
       "const R zv = ddx * ny - ddy * nx;  // along the normal")]),
    ("parabola fit: Cramer numerator with a wrong column",
     [("const R da = T2 * m00 - S3 * u1 + S2 * (T1 * S1 - S2 * T0);",
       "const R da = T2 * m00 - S3 * u1 + S2 * (T1 * S1 - S1 * T0);")]),
    ("fitting frame normal not turned away from the reference phase",
     [("      if (dot > R(0)) {\n        n0x = -n0x;", "      if (dot < R(0)) {\n        n0x = -n0x;")]),
    ("mixed heights measured from the wrong end",
     [("const R pos = o == 1 ? R(-3) + h : R(4) - h;", "const R pos = o == 1 ? R(4) - h : R(-3) + h;")]),
    ("three landings keep the first instead of the middle one",
     [("const Land& m = land[a + n / 2];", "const Land& m = land[a];")]),
    ("three candidates keep the first instead of the middle one",
     [("pick = &cand[a + n / 2];", "pick = &cand[a];")]),
    ("centre rule takes the corner at the other end of the edge",
     [("const int vr = lr < 0 ? -1 : !N.kc(k, lr);",
       "const int vr = lr < 0 ? -1 : !N.kc(k, lr == j ? j + 1 : j);")]),
    ("centre rule walks the right cell in the left column",
     [("const int lr = walk(mB, n4, k);", "const int lr = walk(mB, n4, k - 1);")]),
    ("symmetric difference: clipping keeps the outside",
     [("    if (sc >= 0.0) out.v[out.n++] = cur;", "    if (sc <= 0.0) out.v[out.n++] = cur;")]),
    ("symmetric difference: saddle pieces for the other centre colour",
     [("  if (n == 4 && S.zc(i, j) == 0) {", "  if (n == 4 && S.zc(i, j) == 1) {")]),
    ("markers fit takes vertical markers one edge off",
     [("add((R)(a - i), (R)(b - j) + S.vc(a, b));", "add((R)(a - i) + R(1), (R)(b - j) + S.vc(a, b));")]),
    ("a near neighbour kept as point 1/4 instead of the marker beyond it",
     [("q = local(move(nn), k, j);", "q = local(move(nb), k, j);")]),
    ("chord crossing with the slope's sign flipped",
     [("const double ystar = A.y + (x0 * (B.y - A.y)) / (B.x - A.x);",
       "const double ystar = A.y - (x0 * (B.y - A.y)) / (B.x - A.x);")]),
    ("density law with the phases swapped",
     [("rho[(size_t)j * nx + i] = c * rho1 + (1.0 - c) * rho2;",
       "rho[(size_t)j * nx + i] = (1.0 - c) * rho1 + c * rho2;")]),
    ("face force along minus grad C",
     [("return sigma * kf * (C[b] - C[a]) / dx;", "return sigma * kf * (C[a] - C[b]) / dx;")]),
    ("face curvature drops a lone valid neighbour",
     [("else if (va) kf = ka;", "else if (va) kf = 0.0;")]),
    ("y faces take the cell to the left instead of the one below",
     [("(j == 0 || j == ny) ? 0.0 : face((size_t)(j - 1) * nx + i, (size_t)j * nx + i);",
       "(j == 0 || j == ny) ? 0.0 : face((size_t)j * nx + (i > 0 ? i - 1 : i), (size_t)j * nx + i);")]),
]

BATTERY = [
    (P.test_coupling_properties_pure_phases_and_mass, (0,)),
    (P.test_coupling_flat_interface_has_no_force, ()),
    (P.test_coupling_constant_curvature_telescopes, ()),
    (P.test_coupling_face_curvature_reading, ()),
    (P.test_coupling_laplace_pressure_jump, (True,)),
    (P.test_fit_exact_on_circle, ()),
    (P.test_near_vertex_neighbour_is_passed_over_for_the_next_marker, ()),
    (P.test_fit_collinear_is_the_line_and_degenerate_cases, ()),
    (P.test_translation_table1, (32,)),
    (P.test_aligned_markers_follow_linear_field, (0,)),
    (P.test_aligned_markers_follow_linear_field, (1,)),
    (P.test_straight_line_under_shear_stays_straight, (0,)),
    (P.test_straight_line_under_shear_stays_straight, (1,)),
    (P.test_merge_when_approaching_along_x, ()),
    (P.test_diagonal_approach_keeps_two_loops, ()),
    (P.test_subgrid_drop_disappears, ()),
    (P.test_fraction_exact_for_half_planes, ()),
    (P.test_fraction_saddle_cell_follows_centre_colour, ()),
    (P.test_circle_area_inscribed_polygon_bound, ()),
    (P.test_hf_straight_line_zero_curvature, ()),
    (P.test_hf_circle_curvature_converges, ()),
    (P.test_init_markers_on_shapes, ()),
    (P.test_vortex_T2_table3, (32,)),
    (P.test_three_landings_keep_the_middle_one, ()),
    (P.test_sym_diff_closed_forms, ()),
    (P.test_sym_diff_brute_force, (6,)),
    (P.test_sweep_commutes_with_reflections, ()),
    (P.test_centre_colour_of_saddles_follows_the_exact_shape, ()),
    (P.test_parabola_fit_exact_on_parabolas, ()),
    (P.test_parabola_fit_circle_and_singular, ()),
    (P.test_ghf_keeps_standard_values_and_resolves_packed_disks, (0,)),
    (P.test_ghf_bubbles_negative_and_lines_flat, ()),
]


@pytest.mark.parametrize("name,edits", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, edits, tmp_path):
    src = oracle.source_text()
    for old, new in edits:
        assert src.count(old) == 1, f"mutation site not unique: {old}"
        src = src.replace(old, new)
    lib_path = oracle.compile_variant(src, str(tmp_path / "libmutant.so"))
    failed = []
    with oracle.use_library(lib_path):
        for fn, args in BATTERY:
            try:
                fn(*args)
            except Exception as e:  # AssertionError or a numerical blow-up
                failed.append(fn.__name__)
                break
    assert failed, f"no pin caught the planted mistake: {name}"
