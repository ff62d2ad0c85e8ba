"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check
that the pins in test_oracle_pins.py catch every one of them.

Each mutant is oracle.c with one edit -- a flipped comparison, a dropped
term, a swapped operand -- compiled into a temporary library and driven
through the same Python wrapper in a child process (so a mutant that loops
forever is killed by the timeout instead of hanging the suite).
"""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    # Algorithm 1 threshold: "<=" becomes "<"
    "threshold_strict": ("(u128)deg[v] * q * S <= rhs", "(u128)deg[v] * q * S < rhs"),
    # threshold factor 2(p+q) loses its 2
    "threshold_drop_2": ("u128 rhs = (u128)2 * ((u128)p + q) * E;", "u128 rhs = ((u128)p + q) * E;"),
    # eps = p/q with p and q swapped in the threshold
    "threshold_swap_pq": ("u128 rhs = (u128)2 * ((u128)p + q) * E;", "u128 rhs = (u128)2 * ((u128)q + p) * E * q / (p ? p : 1);"),
    # an edge inside the failed set is counted twice
    "edge_inside_twice": ("} else if (peel_round[u] == r + 1 && u > v) {", "} else if (peel_round[u] == r + 1) {"),
    # an edge inside the failed set is not counted at all
    "edge_inside_dropped": ("} else if (peel_round[u] == r + 1 && u > v) {", "} else if (0) {"),
    # survivor keeps its degree
    "no_decrement": ("deg[u] -= 1;\n                    removed += 1;", "removed += 1;"),
    # failed vertices leave S before the test of the round is complete
    "no_snapshot": ("if (alive[v] && (u128)deg[v] * q * S <= rhs) failed[nf++] = v;",
                    "if (alive[v] && (u128)deg[v] * q * S <= rhs) { failed[nf++] = v; alive[v] = 0; "
                    "for (uint64_t j = off[v]; j < off[v + 1]; ++j) if (alive[adj[j]]) deg[adj[j]]--; }"),
    # keep-best becomes ">="
    "best_nonstrict": ("if (S > 0 && (u128)E * bestV > (u128)bestE * S) {\n            best_round = r;",
                       "if (S > 0 && (u128)E * bestV >= (u128)bestE * S) {\n            best_round = r;"),
    # Batagelj-Zaversnik moves neighbours of equal degree too
    "bz_geq": ("if (d[u] > d[v]) {", "if (d[u] >= d[v]) {"),
    # PKC level scan also picks up vertices finished at earlier levels
    "pkc_scan_leq": ("if (deg[v] == k) buff[end++] = v;", "if (deg[v] <= k) buff[end++] = v;"),
    # ingest keeps self-loops
    "ingest_loops": ("if (u == v) continue;\n        uint64_t lo", "uint64_t lo"),
    # ingest keeps duplicates
    "ingest_dups": ("if (i == 0 || keys[i] != keys[i - 1]) keys[m++] = keys[i];", "keys[m++] = keys[i];"),
    # Goldberg sink capacity with a instead of 2a
    "goldberg_half": ("(int64_t)(m * b + 2 * a) - dv * (int64_t)b", "(int64_t)(m * b + a) - dv * (int64_t)b"),
    # densest-core ties go to the largest k
    "dcore_geq": ("if (!have || (u128)E * out[2] > (u128)out[1] * V)", "if (!have || (u128)E * out[2] >= (u128)out[1] * V)"),
    # phase-2 legit test non-strict
    "cbds_geq": ("if ((u128)cnt * Vk > Ek) { legit[v] = 1;", "if ((u128)cnt * Vk >= Ek) { legit[v] = 1;"),
}

BATTERY = textwrap.dedent("""
    import sys, traceback
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    import ctypes, oracle
    oracle._lib = None
    oracle._LIB_PATH = {lib!r}
    oracle.build = lambda force=False: {lib!r}
    import test_oracle_pins as T
    import pytest
    checks = []
    for name in T.all_fixtures():
        checks.append(lambda name=name: T.test_bahmani_hand_worked(name))
        checks.append(lambda name=name: T.test_kcore_hand_worked(name))
    for name in T.all_fixtures("cbds_"):
        checks.append(lambda name=name: T.test_cbds_hand_worked(name))
    checks += [T.test_canonical_csr_matches_edge_set_brute_force, T.test_two_equal_cliques_keep_round_zero,
               lambda: T.test_star(5), lambda: T.test_complete_graph(7, (1, 10)), lambda: T.test_edgeless(5),
               lambda: T.test_incremental_equals_recompute((1, 10)), lambda: T.test_incremental_equals_recompute((0, 1)),
               T.test_kcore_three_statements_agree, T.test_kcore_matches_networkx, T.test_kcore_invariants,
               lambda: T.test_peel_invariants((1, 10)), T.test_goldberg_matches_brute_force,
               lambda: T.test_bahmani_bound_brute_force((1, 10)), T.test_densest_core_brute_force,
               T.test_cbds_phase2_counts_the_augmented_set]
    failed = 0
    for c in checks:
        try:
            c()
        except BaseException as e:
            failed += 1
    print("FAILED_CHECKS", failed)
""")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(ORACLE_C).read()
    assert before in src, f"mutation anchor for {name} no longer matches oracle.c"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(before, after, 1))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(mut), "-o", str(lib)])
    code = BATTERY.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=str(lib))
    try:
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    except subprocess.TimeoutExpired:
        return  # the pins never finish on this mutant: caught
    lines = [l for l in out.stdout.splitlines() if l.startswith("FAILED_CHECKS")]
    assert lines, out.stderr[-2000:]
    assert int(lines[-1].split()[1]) > 0, f"mutant {name} passed every pin"


def test_unmutated_oracle_passes_battery(tmp_path):
    lib = tmp_path / "liboracle_same.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", ORACLE_C, "-o", str(lib)])
    code = BATTERY.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=str(lib))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert "FAILED_CHECKS 0" in out.stdout, out.stdout + out.stderr[-2000:]
