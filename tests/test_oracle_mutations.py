"""The oracle pins catch plausible mistakes: each case plants one mistake in a
copy of an oracle's C source (a transposed operand, a dropped term, a wrong
sign, a reversed tie-break, a missing correction), builds it, and runs the
pin tests of that oracle against the mutant in a subprocess: they must fail.
A control run of an unmodified copy must pass, so that a failure means the
pins saw the mistake and not a broken harness."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

# source file, environment variable its wrapper reads, the pin tests that cover it
TARGETS = {
    "mesh": ("oracle.c", "ORACLE_MESH_LIB", ["tests/test_oracle_raster.py", "tests/test_oracle_blend.py"]),
    # the same source; its margin flags are covered by their own pins
    "mesh_margins": ("oracle.c", "ORACLE_MESH_LIB", ["tests/test_oracle_margins.py"]),
    "points": ("points.c", "ORACLE_POINTS_LIB", ["tests/test_oracle_points.py"]),
    "shading": ("shading.c", "ORACLE_SHADING_LIB", ["tests/test_oracle_shading.py"]),
    "shading_margins": ("shading.c", "ORACLE_SHADING_LIB", ["tests/test_oracle_shade_margins.py"]),
    "knn": ("knn.c", "ORACLE_KNN_LIB", ["tests/test_oracle_knn.py"]),
}

MUTATIONS = [
    # (target, what the mistake is, original text, mutated text)
    ("mesh", "barycentric edge function with its operands transposed",
     "o->b[0] = orc_edge(v1, v2, px, py) / F->A;", "o->b[0] = orc_edge(v2, v1, px, py) / F->A;"),
    ("mesh", "perspective correction dropped",
     "double t0 = o->b[0] / v0[2], t1 = o->b[1] / v1[2], t2 = o->b[2] / v2[2];",
     "double t0 = o->b[0], t1 = o->b[1], t2 = o->b[2];"),
    ("mesh", "clipped barycentric not renormalised",
     "o->bp[0] = c0 / cs;", "o->bp[0] = c0;"),
    ("mesh", "signed distance with the wrong sign inside",
     "o->d = o->inside ? -o->s : o->s;", "o->d = o->inside ? o->s : -o->s;"),
    ("mesh", "equal depths ordered by descending face id",
     "if (x->f < y->f) return -1;\n    if (x->f > y->f) return 1;",
     "if (x->f > y->f) return -1;\n    if (x->f < y->f) return 1;"),
    # the margin flags the parity tests exclude pixels by
    ("mesh_margins", "margin distance taken squared (flags 1 and 2)",
     "double dist = sqrt(o.s);", "double dist = o.s;"),
    ("mesh_margins", "depth ties looked for in the first pair only (flag 8)",
     "for (int64_t i = 0; i + 1 < m && i < K; i++)", "for (int64_t i = 0; i + 1 < m && i < 1; i++)"),
    ("mesh_margins", "blur boundary flagged inside the face too (flag 2)",
     "if (blur > 0.0 && !o.inside && fabs(dist - rb) < eps) fl |= 2;",
     "if (blur > 0.0 && fabs(dist - rb) < eps) fl |= 2;"),
    ("mesh_margins", "cull-area margin absolute instead of relative (flag 4)",
     "fabs(fabs(Fc.A) - ORC_CULL_AREA) < eps * ORC_CULL_AREA", "fabs(fabs(Fc.A) - ORC_CULL_AREA) < eps"),
    ("mesh_margins", "znear margin of the corners dropped (flag 16)",
     "if (fabs(Fc.P[i][2] - znear) < eps) fl |= 16;", "(void)znear;"),
    ("mesh_margins", "edges meeting at their shared corner counted as a tie (flag 32)",
     "if (a != o.edge && fabs(dd[a] - dd[o.edge]) < eps &&\n                        hypot(nx[a] - nx[o.edge], ny[a] - ny[o.edge]) > eps)",
     "if (a != o.edge && fabs(dd[a] - dd[o.edge]) < eps)"),
    ("mesh_margins", "clip kink flagged without clipping (flag 64)",
     "                if (clip)\n                    for (int a = 0; a < 3; a++)\n                        if (fabs(o.bt[a]) < eps) fl |= 64;",
     "                for (int a = 0; a < 3; a++)\n                        if (fabs(o.bt[a]) < eps) fl |= 64;"),
    ("mesh_margins", "extrapolation weighed by its depth only (flag 128)",
     "if (fabs(o.bt[a]) > mag) mag = fabs(o.bt[a]);", "(void)a;"),
    ("points", "opacity against r instead of r squared",
     "return 1.0 - d / (radius * radius);", "return 1.0 - d / radius;"),
    ("points", "transmittance multiplied by the opacity",
     "T *= 1.0 - a;", "T *= a;"),
    ("shading", "reflection vector with the light term added",
     "const double D = c > 0.0 ? c : 0.0;\n    double r[3];\n    for (int j = 0; j < 3; j++) r[j] = 2.0 * c * m[j] - l[j];",
     "const double D = c > 0.0 ? c : 0.0;\n    double r[3];\n    for (int j = 0; j < 3; j++) r[j] = 2.0 * c * m[j] + l[j];"),
    ("shading", "specular exponent off by one",
     "const double Sp = spec_on ? pow(s, Lt->sh) : 0.0;", "const double Sp = spec_on ? pow(s, Lt->sh - 1.0) : 0.0;"),
    # the kink margin the shading parity tests drop gradients by
    ("shading_margins", "specular switch counted with the light behind the face",
     "if (c > 0.0 && fabs(sv) < mg) mg = fabs(sv);", "if (fabs(sv) < mg) mg = fabs(sv);"),
    ("shading_margins", "diffuse switch dropped from the margin",
     "double mg = fabs(c);", "double mg = 1e300;"),
    ("shading_margins", "hard blend margin taken over every slot",
     "const int64_t kk = blend_mode == 1 ? 1 : K;", "const int64_t kk = K;"),
    ("shading_margins", "Gouraud margin taken at the interpolated point",
     "if (shading == 1) {\n                for (int i = 0; i < 3; i++) {\n                    const double m1",
     "if (shading == 99) {\n                for (int i = 0; i < 3; i++) {\n                    const double m1"),
    ("knn", "the second coordinate's square rounded before the sum (no fma)",
     "s = fmaf(dc, dc, s);", "s = s + dc * dc;"),
    ("knn", "equal distances ranked by descending row",
     "return d < e || (d == e && j < k);", "return d < e || (d == e && j > k);"),
    ("knn", "the first candidate of every cloud skipped",
     "for (int64_t j = first2[i]; j < first2[i] + len2[i]; ++j) {",
     "for (int64_t j = first2[i] + 1; j < first2[i] + len2[i]; ++j) {"),
    ("knn", "the kept list sorted in descending order",
     "while (pos > 0 && ranks_before(d, j, od[pos - 1], oi[pos - 1])) {",
     "while (pos > 0 && ranks_before(od[pos - 1], oi[pos - 1], d, j)) {"),
]


def _run_pins(target, lib_path):
    _, env_name, tests = TARGETS[target]
    env = dict(os.environ, **{env_name: lib_path})
    r = subprocess.run([sys.executable, "-m", "pytest", *tests, "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def _build_variant(target, tmp_path, old=None, new=None):
    src_name = TARGETS[target][0]
    text = open(os.path.join(ORACLE, src_name)).read()
    if old is not None:
        assert text.count(old) == 1, "mutation site not found exactly once: %r" % old
        text = text.replace(old, new)
    return oracle.compile_source(text, str(tmp_path / ("lib_%s.so" % target)))


@pytest.mark.parametrize("target", sorted(TARGETS))
def test_control_copy_passes_its_pins(target, tmp_path):
    rc, out = _run_pins(target, _build_variant(target, tmp_path))
    assert rc == 0, out


@pytest.mark.parametrize("target,what,old,new", MUTATIONS, ids=[m[1] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(target, what, old, new, tmp_path):
    rc, out = _run_pins(target, _build_variant(target, tmp_path, old, new))
    assert rc == 1, "the pins did not catch: %s\n%s" % (what, out)


# the numpy half of the nearest-neighbour oracle (Chamfer loss and gradients):
# the mutant module is swapped in for the pin tests' oracle module in-process
PY_MUTATIONS = [
    ("the Chamfer distance taken as L1 instead of squared L2",
     "np.sum((pts[rows] - other[nn[rows]]) ** 2) / n", "np.sum(np.abs(pts[rows] - other[nn[rows]])) / n"),
    ("the Chamfer gradient without its factor 2",
     "t = 2.0 * g / n * (pts[rows] - other[nn[rows]])", "t = g / n * (pts[rows] - other[nn[rows]])"),
    ("the neighbour's Chamfer gradient with the wrong sign",
     "np.add.at(go, nn[rows], -t)", "np.add.at(go, nn[rows], t)"),
    ("the KNN distance gradient of the neighbour with the wrong sign",
     "np.add.at(g2, idx[rows, k], -t)", "np.add.at(g2, idx[rows, k], t)"),
]


def _numpy_pins_failing(old, new, monkeypatch):
    import types

    import test_oracle_knn as pins
    path = os.path.join(ORACLE, "knn.py")
    text = open(path).read()
    assert text.count(old) == 1, "mutation site not found exactly once: %r" % old
    mutant = types.ModuleType("knn_mutant")
    mutant.__file__ = path
    exec(compile(text.replace(old, new), path, "exec"), mutant.__dict__)
    monkeypatch.setattr(pins, "ok", mutant)
    caught = 0
    for test in (pins.test_chamfer_matches_the_pairwise_matrix_form, pins.test_chamfer_closed_forms,
                 pins.test_chamfer_gradient_matches_central_differences,
                 pins.test_knn_gradient_matches_central_differences):
        try:
            test()
        except AssertionError:
            caught += 1
    return caught


def test_numpy_oracle_control_copy_passes(monkeypatch):
    old = PY_MUTATIONS[0][1]
    assert _numpy_pins_failing(old, old, monkeypatch) == 0


@pytest.mark.parametrize("what,old,new", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_planted_mistake_in_the_numpy_oracle_fails_a_pin(what, old, new, monkeypatch):
    assert _numpy_pins_failing(old, new, monkeypatch) >= 1, "the pins did not catch: %s" % what
