"""Mutation check of the oracle's pins: each mutation below, planted alone
in a copy of the oracle's C source, must make at least one pin fail. They are
the plausible slips the pins are there to catch (a wrong coefficient, weight,
sign, index, table entry, bit width or random word), in the D2Q9 tables, the
D2Q7 tables and streaming, and the step code both lattices share.

Each case copies the oracle, the pin modules and the workload module into
_build/mut/<case> at the repository root (git-ignored; not under tests/, whose
conftest would put the repository's own oracle first on the path), rebuilds
the oracle there and runs the pins in a subprocess, the mutated lattice's
first."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_invariants.py", "tests/test_oracle_philox.py",
        "tests/test_oracle_d2q7.py", "tests/test_oracle_d2q7_growth.py"]

MUTANTS = [
    ("c1 3 -> 2.5", "    3.0, 4.5, 1.5,", "    2.5, 4.5, 1.5,"),
    ("c2 4.5 -> 4", "    3.0, 4.5, 1.5,", "    3.0, 4.0, 1.5,"),
    ("c3 1.5 -> 1", "    3.0, 4.5, 1.5,", "    3.0, 4.5, 1.0,"),
    ("w0", "{4.0 / 9.0, 1.0 / 9.0,", "{0.45, 1.0 / 9.0,"),
    ("w8", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0},", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 30.0},"),
    ("opp table", "{0, 3, 4, 1, 2, 7, 8, 5, 6},", "{0, 3, 4, 1, 2, 8, 7, 6, 5},"),
    ("pair table", "{1, 2, 5, 6},\n    {3, 4, 7, 8}};", "{1, 2, 5, 6},\n    {3, 4, 8, 7}};"),
    ("jx sign", "*jx = ((((fs[1] - fs[3]) + fs[5]) - fs[6])", "*jx = ((((fs[1] - fs[3]) + fs[5]) + fs[6])"),
    ("jy sign", "+ fs[6]) - fs[7]) - fs[8];", "+ fs[6]) - fs[7]) + fs[8];"),
    ("stream x", "*xs = x - (int)s->L->ex[i];", "*xs = x + (int)s->L->ex[i];"),
    ("stream y", "*ys = y - (int)s->L->ey[i];", "*ys = y + (int)s->L->ey[i];"),
    ("friction sign", "const double cmu = 1.0 - s->p.mu;", "const double cmu = 1.0 + s->p.mu;"),
    ("BGK sign", "fo[i] = fs[i] - omega * (fs[i] - fss);", "fo[i] = fs[i] + omega * (fs[i] - fss);"),
    ("noise mean", "const double ubar = S / (double)Q;", "const double ubar = S / (double)(Q - 1);"),
    ("fix adds 2a", "fo[L->opp[i]] = fo[L->opp[i]] + a;", "fo[L->opp[i]] = fo[L->opp[i]] + 2.0 * a;"),
    ("clip ledger", "s->st.clip_mass += 2.0 * a;", "s->st.clip_mass += a;"),
    ("carry dropped", "s->st.carry = x_ns - fl;", "s->st.carry = 0.0;"),
    ("edge depth <", "(s->h[x] - y) <= s->p.edge_depth", "(s->h[x] - y) < s->p.edge_depth"),
    ("Eq. 5 inverted", "u01(r[2]) < 1.0 - rs / s->p.rho0", "u01(r[2]) < rs / s->p.rho0"),
    ("wall factor", "double wg = s->p.wall_w_factor * s->st.w;", "double wg = s->st.w;"),
    ("height off by one", "hx = y + 1; /* h(x) = 1 + highest occupied row */", "hx = y; /* h(x) = 1 + highest occupied row */"),
    ("half cell", "const double half = s->p.rho_cell * 0.5;", "const double half = s->p.rho_cell * 0.25;"),
    ("pair word", "(int)(r[1] >> 30)", "(int)(r[2] >> 30)"),
    ("node word", "(((uint64_t)r[0] * (uint64_t)nwin) >> 32)", "(((uint64_t)r[3] * (uint64_t)nwin) >> 32)"),
    ("band + 1", "if (yr + s->p.band_rows < y_hi) y_hi = yr + s->p.band_rows;",
     "if (yr + s->p.band_rows + 1 < y_hi) y_hi = yr + s->p.band_rows + 1;"),
    # D2Q7
    ("D2Q7 q2 parity shift", "case 2: *xs = x - 1 + par; *ys = y - 1;", "case 2: *xs = x - par; *ys = y - 1;"),
    ("D2Q7 q3 parity shift", "case 3: *xs = x + par; *ys = y - 1;", "case 3: *xs = x + 1 - par; *ys = y - 1;"),
    ("D2Q7 q5 row", "case 5: *xs = x + par; *ys = y + 1;", "case 5: *xs = x + par; *ys = y - 1;"),
    ("D2Q7 c1 4 -> 3", "    4.0, 8.0, 2.0,", "    3.0, 8.0, 2.0,"),
    ("D2Q7 c2 8 -> 9", "    4.0, 8.0, 2.0,", "    4.0, 9.0, 2.0,"),
    ("D2Q7 c3 2 -> 1.5", "    4.0, 8.0, 2.0,", "    4.0, 8.0, 1.5,"),
    ("D2Q7 w0 0.5 -> 0.4", "    {0.5, 1.0 / 12.0,", "    {0.4, 1.0 / 12.0,"),
    ("D2Q7 opp table", "    {0, 4, 5, 6, 1, 2, 3},", "    {0, 4, 6, 5, 1, 3, 2},"),
    ("D2Q7 pair table", "    {1, 2, 3},\n    {4, 5, 6}};", "    {1, 2, 3},\n    {4, 6, 5}};"),
    ("D2Q7 jx sign", "+ 0.5 * fs[2]) - 0.5 * fs[3])", "- 0.5 * fs[2]) - 0.5 * fs[3])"),
    ("D2Q7 jy factor", "- fs[6]) * HALF_SQRT3;", "- fs[6]) * 0.5;"),
    ("D2Q7 fbits 18 -> 17", "    7, 3, 18,", "    7, 3, 17,"),
    ("D2Q7 pair draw", "(((uint64_t)r[1] * (uint64_t)L->npairs) >> 32)", "(((uint64_t)r[1] * (uint64_t)2) >> 32)"),
    ("D2Q7 ex2 sign", "    {0.0, 1.0, 0.5, -0.5, -1.0, -0.5, 0.5},", "    {0.0, 1.0, -0.5, -0.5, -1.0, -0.5, 0.5},"),
    ("D2Q7 ey5 sign", "    {0.0, 0.0, HALF_SQRT3, HALF_SQRT3, 0.0, -HALF_SQRT3, -HALF_SQRT3},",
     "    {0.0, 0.0, HALF_SQRT3, HALF_SQRT3, 0.0, HALF_SQRT3, -HALF_SQRT3},"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mutation(name, old, new):
    src = open(os.path.join(ROOT, "oracle", "lbm_oracle.c")).read()
    assert src.count(old) == 1, f"mutation site of {name!r} not found once"
    work = os.path.join(ROOT, "_build", "mut", name.replace(" ", "_").replace(">", "").replace(".", ""))
    shutil.rmtree(work, ignore_errors=True)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(work, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__", "*.so"))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(work, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__", "_build"))
    os.makedirs(os.path.join(work, "paper_2303_02210_gb300"))
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_2303_02210_gb300", f), os.path.join(work, "paper_2303_02210_gb300", f))
    with open(os.path.join(work, "oracle", "lbm_oracle.c"), "w") as fh:
        fh.write(src.replace(old, new))
    try:
        pins = PINS[2:] + PINS[:2] if name.startswith("D2Q7") else PINS
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *pins],
                           cwd=work, capture_output=True, text=True, timeout=900)
    finally:
        shutil.rmtree(work, ignore_errors=True)
    assert r.returncode == 1, f"{name}: the pins did not fail (rc {r.returncode})\n{r.stdout[-1500:]}"
