"""Plant plausible mistakes in copies of the oracle (on the CPU) and check that the
pins of test_oracle_pins.py catch every one of them."""
import os

import numpy as np
import pytest

import test_oracle_pins as pins
from oracle import oracle as O
from paper_2208_14567_gb300 import inputs as I

MUTANTS = {
    "swapped lengths in e": ("double e = d2 + P->r1sq[d] - P->r2sq[d];", "double e = d2 - P->r1sq[d] + P->r2sq[d];"),
    "wrong length in D": ("double D = 4.0 * d2 * P->r1sq[d] - e * e;", "double D = 4.0 * d2 * P->r2sq[d] - e * e;"),
    "wrong branch": ("double sh = (double)P->s[d] * h;", "double sh = -(double)P->s[d] * h;"),
    "dropped perpendicular term": ("out[2 * P->k[d]] = pi[0] + (e * dx - sh * dy) * inv;",
                                   "out[2 * P->k[d]] = pi[0] + (e * dx) * inv;"),
    "clockwise crank": ("out[2 * P->motor + 1] = pv[1] + (s * ux + c * uy);",
                        "out[2 * P->motor + 1] = pv[1] + (-s * ux + c * uy);"),
    "never locks": ("if (!(q > 0.0)) {", "if (q < -1e300) {"),
    "branch sign flipped": ("P->s[nd] = cross < 0.0 ? -1 : 1;", "P->s[nd] = cross > 0.0 ? -1 : 1;"),
    "highest ready joint first": ("if (cnt >= 2) { pick = a; break; }", "if (cnt >= 2) { pick = a; }"),
    "no edge-count check": ("if (links != 2 * n_simple) return P->status = LO_OVERCONSTRAINED;", ""),
    "normalise sign rule flipped": ("if (s3 < 0.0)", "if (s3 > 0.0)"),
    "squared chamfer": ("double d = sqrt(sq_dist(P + 2 * a, Q + 2 * b));", "double d = sq_dist(P + 2 * a, Q + 2 * b);"),
    "one-directional chamfer": ("return sp / tp + sq / tq;", "return sp / tp;"),
    "max line rotated the wrong way": ("double xr = (c * x + s * y) / d, yr = (-s * x + c * y) / d;",
                                       "double xr = (c * x - s * y) / d, yr = (s * x + c * y) / d;"),
    "max line not scaled": ("double xr = (c * x + s * y) / d, yr = (-s * x + c * y) / d;",
                            "double xr = (c * x + s * y), yr = (-s * x + c * y);"),
    "max line centred at the first point": ("double sx = 0.5 - 0.5 * (x0 + x1), sy = 0.5 - 0.5 * (y0 + y1);",
                                            "double sx = 0.0, sy = 0.5;"),
    "max line pair not the farthest": ("if (d > best) { best = d; a = u; b = v; }",
                                       "if (d > best && v == u + 1) { best = d; a = u; b = v; }"),
    "circle variance of squared radii": ("m2 += r * r;", "m2 += r * r * r * r;"),
    # the margin indicator q = D / (4 r1^2 r2^2) and its running minima
    "q with r1 squared twice": ("double q = D / (4.0 * P->r1sq[d] * P->r2sq[d]);",
                                "double q = D / (4.0 * P->r1sq[d] * P->r1sq[d]);"),
    "min |q| skips the locking dyad": ("        double aq = fabs(q);\n        if (aq < qabs || aq != aq) qabs = aq;\n"
                                       "        if (!(q > 0.0)) {",
                                       "        double aq = fabs(q);\n        if (!(q > 0.0)) {"),
    "min q includes the locking step": ("            if (locked) { lock = t; break; }\n"
                                        "            if (qmin < qmin_all) qmin_all = qmin;",
                                        "            if (qmin < qmin_all) qmin_all = qmin;\n"
                                        "            if (locked) { lock = t; break; }"),
    "min |q| skips the locking step": ("            if (qabs < qabs_all || qabs != qabs) qabs_all = qabs;\n"
                                       "            if (locked) { lock = t; break; }",
                                       "            if (locked) { lock = t; break; }\n"
                                       "            if (qabs < qabs_all || qabs != qabs) qabs_all = qabs;"),
}


def run_pins(lib):
    """Every pin of test_oracle_pins.py with this oracle build; returns the failures."""
    saved = O._lib
    O._lib = lib
    failures = []
    try:
        f = I.fourbar_batch(400, seed=0)
        d = I.dyad_batch(600, 6, 12, seed=1, permute=True)
        fourbars = (f, O.simulate(f, pins.T))
        dyads = (d, O.simulate(d, pins.T))
        checks = [
            lambda: pins.test_plan_fourbar(O),
            lambda: pins.test_plan_solve_order_follows_lowest_ready_joint(O),
            lambda: pins.test_extra_link_breaks_mobility_and_plan(O),
            lambda: pins.test_step0_reproduces_initial_positions(fourbars, dyads),
            lambda: pins.test_rigidity_every_link_keeps_its_length(dyads, fourbars),
            lambda: pins.test_nan_from_lock_and_flags(dyads),
            lambda: pins.test_closure_at_full_turn(O, dyads),
            lambda: pins.test_fourbar_matches_trigonometric_solution(fourbars),
            lambda: pins.test_fourbar_margin_indicator_closed_form(fourbars),
            lambda: pins.test_margin_indicator_from_positions(O, dyads),
            lambda: pins.test_full_rotation_criterion(fourbars),
            lambda: pins.test_brute_force_branches(O),
            lambda: pins.test_special_cases(O),
            lambda: pins.test_normalize_properties_and_invariance(O, fourbars),
            lambda: pins.test_normalize_ellipse_and_degenerate(O),
            lambda: pins.test_chamfer_against_cdist(O),
            lambda: pins.test_maxline_circle_ellipse_segment(O),
            lambda: pins.test_maxline_pair_is_the_farthest_pair(O),
            lambda: pins.test_maxline_similarity_invariance_and_mirror(O),
            lambda: pins.test_maxline_degenerate_and_imposed_pair(O),
        ]
        for i, c in enumerate(checks):
            try:
                c()
            except (AssertionError, ValueError, IndexError, ZeroDivisionError, TypeError):
                failures.append(i)
    finally:
        O._lib = saved
    return failures


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = O.source()
    assert src.count(old) == 1, f"mutation site not found: {old}"
    lib = O.compile_variant(src.replace(old, new), os.path.join(str(tmp_path), "mutant.so"))
    assert run_pins(lib), f"no pin caught the mutant '{name}'"


def test_unmutated_oracle_passes_all(tmp_path):
    lib = O.compile_variant(O.source(), os.path.join(str(tmp_path), "same.so"))
    assert run_pins(lib) == []


# Mistakes planted in the oracle's Python functions (the paper's retrieval and curation,
# and the keep draws' generator): the function's source with one replacement, run in
# the oracle module's namespace, must fail one of the pins that cover it.
PY_MUTANTS = {
    "scan in index order": ("first_under", "hits = order[dist[order] < threshold][:k]",
                            "hits = np.sort(order[dist[order] < threshold])[:k]"),
    "cut-off inclusive": ("first_under", "hits = order[dist[order] < threshold][:k]",
                          "hits = order[dist[order] <= threshold][:k]"),
    "arc when linked to any joint": ("curate_paths", "arc = any(batch.adj[b, j, k] and batch.jtype[b, k] == 0 for k in range(n))",
                                     "arc = any(batch.adj[b, j, k] for k in range(n))"),
    "circle test reversed": ("curate_paths", "circle = var[0] < circle_var", "circle = var[0] > circle_var"),
    "arcs and circles always kept": ("curate_paths", "kept = not (arc or circle) or u < keep_rate",
                                     "kept = not (arc or circle) or u <= 1.0"),
    "generator constant": ("splitmix64", "0xBF58476D1CE4E5B9", "0xBF58476D1CE4E5B7"),
}


def _mutated_oracle(fn_name, old, new):
    import inspect
    import types
    src = inspect.getsource(getattr(O, fn_name))
    assert src.count(old) == 1, (fn_name, old)
    ns = dict(vars(O))
    exec(compile(src.replace(old, new), f"<mutant {fn_name}>", "exec"), ns)
    mod = types.SimpleNamespace(**{k: v for k, v in vars(O).items() if not k.startswith("__")})
    setattr(mod, fn_name, ns[fn_name])
    # functions that call the mutated one must see it too
    for name in ("chamfer_first_under", "curate_paths"):
        if name != fn_name:
            f = ns[name] if name in ns else getattr(O, name)
            g = types.FunctionType(f.__code__, ns, f.__name__, f.__defaults__, f.__closure__)
            setattr(mod, name, g)
    ns.update({fn_name: ns[fn_name]})
    return mod


@pytest.mark.parametrize("name", sorted(PY_MUTANTS))
def test_pins_catch_python_mutant(name):
    fn_name, old, new = PY_MUTANTS[name]
    mod = _mutated_oracle(fn_name, old, new)
    checks = [lambda: pins.test_first_under_scan_order(mod), lambda: pins.test_curation_flags(mod),
              lambda: pins.test_splitmix64_published_outputs(mod)]
    caught = 0
    for c in checks:
        try:
            c()
        except AssertionError:
            caught += 1
    assert caught > 0, f"no pin catches the mutant '{name}'"


def test_python_mutation_harness_control():
    """The unmutated functions, run through the same harness, pass every pin."""
    for fn_name, old, _ in PY_MUTANTS.values():
        mod = _mutated_oracle(fn_name, old, old)
        pins.test_first_under_scan_order(mod)
        pins.test_curation_flags(mod)
        pins.test_splitmix64_published_outputs(mod)
