"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a sign, a
dropped term, a swapped operand, a wrong index or bound, an off-by-one in a
limit or a tie-break), builds it the way the oracle is built, and runs the
fast pins of tests/oracle_checks.py against it in a child process (the
library is chosen through ORACLE_LIB). The numpy layer of the oracle (the
gradient, the entry points, interaction sampling, the loss, the CSR lists)
gets the same treatment: a copy of the package with one change is imported
in place of the real one (ORACLE_PKG), over the unchanged C library. Every
mutant must fail at least one pin; the unchanged sources must pass them
all. CPU only.

One plausible change is left out because no pin can see it: removing the
clamp of a negative numerator (reading R3). The numerator of a plane ahead
rounds below zero only when the point lies on that plane to within rounding,
and the unclamped step then moves the point back by a rounding error.
"""
import concurrent.futures
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "voronoi_oracle.c")
PY_SRC = os.path.join(ROOT, "oracle", "__init__.py")

# (name, text in the source, its replacement); each text occurs exactly once
MUTANTS = [
    ("normal sign, Eq. 1", "for (int c = 0; c < 3; c++) n[c] = pj[c] - pm[c];          /* Eq. 1 */",
     "for (int c = 0; c < 3; c++) n[c] = pm[c] - pj[c];          /* Eq. 1 */"),
    ("midpoint without the half, Eq. 2", "mid[c] = (pj[c] + pm[c]) * 0.5; /* Eq. 2 */", "mid[c] = (pj[c] + pm[c]); /* Eq. 2 */"),
    ("numerator operands swapped, Eq. 4", "for (int c = 0; c < 3; c++) w[c] = mid[c] - r[c];",
     "for (int c = 0; c < 3; c++) w[c] = r[c] - mid[c];"),
    ("facing test inverted, R2", "if (!(den > 0.0)) return 0;                                 /* R2 */",
     "if (!(den < 0.0)) return 0;                                 /* R2 */"),
    ("wall bounds swapped, Eq. 5", "double bound = hi ? X->box[3 + axis] : X->box[axis];",
     "double bound = hi ? X->box[axis] : X->box[3 + axis];"),
    ("tie to the higher id, R4", "if (s < best || (s == best && j < best_id)) {",
     "if (s < best || (s == best && j > best_id)) {"),
    ("zero-length segments emitted, R5", "        if (best > 0.0) {\n            if (ns < X->cap) {",
     "        if (best >= 0.0) {\n            if (ns < X->cap) {"),
    ("density of the next cell in tau", "tau += X->kappa * X->rho[m] * best;",
     "tau += X->kappa * X->rho[best_id < 0 ? m : best_id] * best;"),
    ("point update with a transposed index, R9", "for (int c = 0; c < 3; c++) r[c] = r[c] + best * k[c];  /* R9 */",
     "for (int c = 0; c < 3; c++) r[c] = r[c] + best * k[(c + 1) % 3];  /* R9 */"),
    ("nudge backwards when no exit is found",
     "/* no exit found: nudge over epsilon and relocate (Sect. 2.2) */\n            nfb++;\n"
     "            for (int c = 0; c < 3; c++) r[c] = r[c] + X->eps_nudge * k[c];",
     "/* no exit found: nudge over epsilon and relocate (Sect. 2.2) */\n            nfb++;\n"
     "            for (int c = 0; c < 3; c++) r[c] = r[c] - X->eps_nudge * k[c];"),
    ("zero-run limit off by one", "if (zrun > X->zmax) {", "if (zrun >= X->zmax) {"),
    ("epsilon from the summed extents, R6", "X.eps_nudge = 1e-12 * sqrt(dx * dx + dy * dy + dz * dz); /* R6 */",
     "X.eps_nudge = 1e-12 * (dx + dy + dz); /* R6 */"),
    ("locate ties to the higher index", "if (d2 < bd) { sd = bd; bd = d2; best = j; }",
     "if (d2 <= bd) { sd = bd; bd = d2; best = j; }"),
    ("security radius too small", "if (!X->brute && dist > 2.0 * rmax + 4.0 * X->eps) { stopped = 1; break; }",
     "if (!X->brute && dist > 1.0 * rmax + 4.0 * X->eps) { stopped = 1; break; }"),
    ("clipping plane off the midpoint in z",
     "double mid[3] = {0.5 * (pj[0] + pm[0]), 0.5 * (pj[1] + pm[1]), 0.5 * (pj[2] + pm[2])};",
     "double mid[3] = {0.5 * (pj[0] + pm[0]), 0.5 * (pj[1] + pm[1]), 0.5 * (pj[2] + pm[2]) + 1e-3};"),
    ("pyramid volume with 1/2", "vol += a * h / 3.0;", "vol += a * h / 2.0;"),
    ("small faces dropped from the lists", "        if (a > X->area_tol) {", "        if (a > 1e-3) {"),
    ("sphere exit takes the wrong root", "double s = b > 0.0 ? -q / (b + sq) : sq - b;",
     "double s = b > 0.0 ? -q / (b + sq) : -sq - b;"),
    ("sphere exit without the z term",
     "double q = ((o[0] * o[0] + o[1] * o[1]) + o[2] * o[2]) - sph[3] * sph[3];",
     "double q = (o[0] * o[0] + o[1] * o[1]) - sph[3] * sph[3];"),
    ("open ball instead of closed", "if (!((dx * dx + dy * dy) + dz * dz <= sph[3] * sph[3])) return 0;",
     "if (!((dx * dx + dy * dy) + dz * dz < sph[3] * sph[3])) return 0;"),
]

# the same for the numpy layer (oracle/__init__.py)
PY_MUTANTS = [
    ("gradient without kappa", "w = (dL[:, None] * kappa * tr.seg_len)[mask]", "w = (dL[:, None] * tr.seg_len)[mask]"),
    ("slab entry from the far plane", "t_in = max(t_in, min(t1, t2))", "t_in = max(t_in, max(t1, t2))"),
    ("box test passes with one axis inside", "if np.all((r >= box[:3]) & (r <= box[3:])):",
     "if np.any((r >= box[:3]) & (r <= box[3:])):"),
    ("sphere entry at the far root", "t = q / (np.sqrt(disc) - b) + eps", "t = (np.sqrt(disc) - b) + eps"),
    ("sphere entry without the epsilon", "t = q / (np.sqrt(disc) - b) + eps", "t = q / (np.sqrt(disc) - b)"),
    ("epsilon from the summed extents, numpy layer", "return 1e-12 * float(np.linalg.norm(box[3:] - box[:3]))",
     "return 1e-12 * float(np.sum(box[3:] - box[:3]))"),
    ("interaction distance without 1/(kappa rho)", "s[i] = dist + (part / k if k > 0 else 0.0)",
     "s[i] = dist + part"),
    ("absorption not capped at tau_int", "absorbed[c] += w[i] * (np.exp(-tau) - np.exp(-ti[i]))",
     "absorbed[c] += w[i] * (np.exp(-tau) - np.exp(-(tau + d)))"),
    ("absorption without the weight", "absorbed[c] += w[i] * (np.exp(-tau) - np.exp(-(tau + d)))",
     "absorbed[c] += (np.exp(-tau) - np.exp(-(tau + d)))"),
    ("running distance not advanced", "            dist += l\n", ""),
    ("loss derivative without the chain factor", "-2.0 * (e - t) * e", "-2.0 * (e - t)"),
    ("loss derivative with the wrong sign", "-2.0 * (e - t) * e", "2.0 * (e - t) * e"),
    ("CSR offsets shifted by one", "np.cumsum(deg, out=off[1:])", "np.cumsum(deg, out=off[:-1])"),
    ("a ray's segments cut one short", "return self.seg_cell[i, :n], self.seg_len[i, :n]",
     "return self.seg_cell[i, :n - 1], self.seg_len[i, :n - 1]"),
    ("gradient summed over one segment too many", "mask = np.arange(cap)[None, :] < tr.nseg[:, None]",
     "mask = np.arange(cap)[None, :] <= tr.nseg[:, None]"),
]


def _run_checks(lib, pkg=None):
    env = dict(os.environ, ORACLE_LIB=lib, ORACLE_THREADS="1")
    env.pop("ORACLE_PKG", None)
    if pkg:
        env["ORACLE_PKG"] = pkg
    return subprocess.run([sys.executable, "-m", "tests.oracle_checks"], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=600)


def _py_check(tmpdir, name, text, lib):
    pkg = os.path.join(tmpdir, name)
    os.makedirs(os.path.join(pkg, "oracle"))
    with open(os.path.join(pkg, "oracle", "__init__.py"), "w") as f:
        f.write(text)
    return _run_checks(lib, pkg)


def _build_and_check(tmpdir, name, text):
    src = os.path.join(tmpdir, f"{name}.c")
    with open(src, "w") as f:
        f.write(text)
    lib = os.path.join(tmpdir, f"{name}.so")
    subprocess.check_call(oracle.compile_command(src, lib))
    return _run_checks(lib)


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    """Every mutant and the unchanged source, built and checked in parallel."""
    tmpdir = str(tmp_path_factory.mktemp("mutants"))
    src = open(SRC).read()
    jobs = {"control": src}
    for i, (name, old, new) in enumerate(MUTANTS):
        assert src.count(old) == 1, f"mutation site not found once: {name}"
        jobs[name] = src.replace(old, new)
    py = open(PY_SRC).read()
    py_jobs = {"py control": py}
    for name, old, new in PY_MUTANTS:
        assert py.count(old) == 1, f"mutation site not found once: {name}"
        py_jobs[name] = py.replace(old, new)
    lib = os.path.join(tmpdir, "control.so")
    subprocess.check_call(oracle.compile_command(SRC, lib))
    workers = max(2, min(len(jobs) + len(py_jobs), os.cpu_count() or 2))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        futs = {name: ex.submit(_build_and_check, tmpdir, f"m{i}", text) for i, (name, text) in enumerate(jobs.items())}
        futs.update({name: ex.submit(_py_check, tmpdir, f"p{i}", text, lib) for i, (name, text) in enumerate(py_jobs.items())})
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.parametrize("name", ["control", "py control"])
def test_unchanged_oracle_passes_the_checks(results, name):
    r = results[name]
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS + PY_MUTANTS])
def test_planted_mistake_is_caught(results, name):
    r = results[name]
    assert r.returncode != 0, f"no pin failed for: {name}\n{r.stdout}"
