"""Plant one plausible mistake at a time in a copy of the oracle source and
require that at least one pin catches it.  This shows the pins would notice
a dropped term, a wrong sign or index, a flipped comparison, an off-by-one in
the NPDU window or the sector bounds, and a wrong tie-break."""
import os

import pytest

import oracle
import oracle_pins

# (name, text in the oracle source, replacement, which occurrence: 0 = first)
MUTANTS = [
    ("f32_drop_dy", "float dist = (dx * dx + dy * dy) + dz * dz;", "float dist = (dx * dx) + dz * dz;", 0),
    ("f32_drop_dz", "float dist = (dx * dx + dy * dy) + dz * dz;", "float dist = (dx * dx + dy * dy);", 0),
    ("f32_sign_dy", "float dy = P[3 * j + 1] - py;", "float dy = P[3 * j + 1] + py;", 0),
    ("f32_index_dz", "float dz = P[3 * j + 2] - pz;", "float dz = P[3 * j + 1] - pz;", 0),
    ("f32_swap_operand", "const float py = P[3 * p + 1];", "const float py = P[3 * p + 0];", 0),
    ("f32_update_max", "if (dist <= D[j]) D[j] = dist;", "if (dist >= D[j]) D[j] = dist;", 0),
    ("f32_tie_highest", "if (D[j] > D[best]) best = j;", "if (D[j] >= D[best]) best = j;", 0),
    ("f32_argmin", "if (D[j] > D[best]) best = j;", "if (D[j] < D[best]) best = j;", 0),
    ("f32_scan_from_1", "int64_t best = 0;", "int64_t best = 1;", 0),
    ("window_right", "*kr = k - k / 2;", "*kr = k / 2;", 0),
    ("window_left", "*kl = k / 2;", "*kl = k - k / 2;", 0),
    ("window_has_sample", "*kr = (k - 1) - (k - 1) / 2;", "*kr = k - (k - 1) / 2;", 0),
    ("full_first_ignored", "if (k > 0 && !(full_first && t == 0)) {", "if (k > 0) {", 0),
    ("full_first_every_time", "if (k > 0 && !(full_first && t == 0)) {", "if (k > 0 && !full_first) {", 0),
    ("f32_window_shift", "if (a < 0) a = 0;", "if (a < 0) { b = b - a; a = 0; }", 0),
    ("f32_init", "#define ORACLE_DIST_INIT_F32 1e10f", "#define ORACLE_DIST_INIT_F32 0.5f", 0),
    ("f32_local_index", "out[t] = (int32_t)(lo + p);", "out[t] = (int32_t)(p);", 0),
    ("f64_drop_dy", "double dist = (dx * dx + dy * dy) + dz * dz;", "double dist = (dx * dx) + dz * dz;", 0),
    ("f64_tie_highest", "if (D[j] > D[best]) best = j;", "if (D[j] >= D[best]) best = j;", 1),
    ("f64_update_max", "if (dist <= D[j]) D[j] = dist;", "if (dist >= D[j]) D[j] = dist;", 1),
    ("sector_ceil", "int64_t lo1 = ((s + 1) * N) / M;", "int64_t lo1 = ((s + 1) * N + M - 1) / M;", 0),
    ("samples_ceil", "int64_t off1 = ((s + 1) * C) / M;", "int64_t off1 = ((s + 1) * C + M - 1) / M;", 0),
    ("start_ignored", "int64_t first = r < n - 1 ? r : n - 1;\n        oracle_sector_fps_f32",
     "int64_t first = 0;\n        oracle_sector_fps_f32", 0),
    ("start_unclipped", "first[s] = l + (r < n - 1 ? r : n - 1);", "first[s] = l + r;", 0),
    ("too_small_unchecked", "if (c > n) return ORACLE_ERR_SECTOR_TOO_SMALL;", "", 0),
    ("coverage_max", "if (d < best) best = d;", "if (d > best && best != INFINITY) best = d;", 0),
    ("ball_le", "if (d2 < r2) out", "if (d2 <= r2) out", 0),
    ("ball_pad_last", "const int32_t fill = cnt > 0 ? out[(int64_t)s * K] : -1;",
     "const int32_t fill = cnt > 0 ? out[(int64_t)s * K + cnt - 1] : -1;", 0),
    ("ball_drop_dz", "float d2 = (dx * dx + dy * dy) + dz * dz;", "float d2 = (dx * dx + dy * dy);", 0),
    ("knn_tie_high", "return (x->j > y->j) - (x->j < y->j);", "return (x->j < y->j) - (x->j > y->j);", 0),
    ("knn_drop_dz", "keys[j].d = (ex * ex + ey * ey) + ez * ez;", "keys[j].d = (ex * ex + ey * ey);", 0),
    ("knn_sign_ey", "float ey = xyz[3 * j + 1] - cy;", "float ey = xyz[3 * j + 1] + cy;", 0),
    ("knn_farthest", "if (x->d < y->d) return -1;\n    if (x->d > y->d) return 1;",
     "if (x->d < y->d) return 1;\n    if (x->d > y->d) return -1;", 0),
]


def _mutate(text, old, new, occurrence):
    pos = -1
    for _ in range(occurrence + 1):
        pos = text.find(old, pos + 1)
        assert pos >= 0, f"mutation site not found: {old!r}"
    return text[:pos] + new + text[pos + len(old):]


@pytest.mark.parametrize("name,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new, occ):
    with open(oracle.SOURCE) as f:
        src = f.read()
    mutated = _mutate(src, old, new, occ)
    assert mutated != src
    c_path = os.path.join(tmp_path, "mutant.c")
    with open(c_path, "w") as f:
        f.write(mutated)
    lib_path = oracle.compile_oracle(c_path, os.path.join(tmp_path, f"lib_{name}.so"), werror=False)
    L = oracle.load_library(lib_path)
    failed = []
    for pin in oracle_pins.PINS:
        try:
            pin(L)
        except (AssertionError, oracle.OracleError, ValueError, IndexError):
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"
