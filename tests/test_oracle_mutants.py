"""Planted mistakes in the oracle must each fail at least one pin.

Every mutant is one textual edit of a copy of oracle/vg_oracle.c (a dropped
term, a wrong sign, index or tie-break, a transposed operand ...), built with
the oracle's own flags into a temporary directory and run against all checks
of oracle_pins.py in a child process.  Nothing here touches the CUDA path.
"""
import json
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "vg_oracle.c")

MUTANTS = {
    "tie_break_highest_axis": ("if (tmax[1] < tmax[m]) m = 1;", "if (tmax[1] <= tmax[m]) m = 1;"),
    "boundary_off_by_one": ("float b = (float)(step[k] > 0 ? i[k] + 1 : i[k]);",
                            "float b = (float)(step[k] > 0 ? i[k] : i[k]);"),
    "ray_too_short": ("if (!(tmax[m] < 1.0f)) break;", "if (!(tmax[m] < 0.9f)) break;"),
    "dropped_translation": ("g = g + T->t[k];", "g = g + 0.0f * T->t[k];"),
    "transposed_rotation": ("float g = T->R[k * 3 + 0] * x + T->R[k * 3 + 1] * y;\n"
                            "        g = g + T->R[k * 3 + 2] * z;",
                            "float g = T->R[0 * 3 + k] * x + T->R[1 * 3 + k] * y;\n"
                            "        g = g + T->R[2 * 3 + k] * z;"),
    "inflate_radius_plus_one": ("stamp_cube(n, c, p->vox_inf, occ_inf);",
                                "stamp_cube(n, c, p->vox_inf + 1, occ_inf);"),
    "traced_beats_free": ("else if (fr[i]) ms[i] = OR_FREE;\n        else if (tr[i]) ms[i] = OR_TRACED;",
                          "else if (tr[i]) ms[i] = OR_TRACED;\n        else if (fr[i]) ms[i] = OR_FREE;"),
    "index_strides_swapped": ("return (int64_t)x + (int64_t)n[0] * ((int64_t)y + (int64_t)n[1] * z);",
                              "return (int64_t)x + (int64_t)n[1] * ((int64_t)y + (int64_t)n[0] * z);"),
    "shift_sign": ("int32_t sx = x + delta[0], sy = y + delta[1], sz = z + delta[2];",
                   "int32_t sx = x - delta[0], sy = y - delta[1], sz = z - delta[2];"),
    "rays_see_raw_occupancy": ("const uint8_t *tested = occ_inf;", "const uint8_t *tested = occ_raw;"),
    "principal_point_w_over_2": ("K[2] = (float)(((double)W - 1.0) / 2.0);",
                                 "K[2] = (float)((double)W / 2.0);"),
    "never_traced": ("R->traced = 1;", "R->traced = 0;"),
    "step_sign_ignored": ("step[k] = D[k] > 0.0f ? 1 : -1;", "step[k] = 1;"),
    "u16_scale_ignored": ("d = (float)raw * scale;", "d = (float)raw;"),
    "no_range_filter": ("if (!(isfinite(d) && d > 0.0f && d <= p->depth)) return 0;",
                        "if (!(isfinite(d) && d > 0.0f)) return 0;"),
    "half_width_truncated": ("long hw = lround(tan(half_fov_rad(p->fov_x_deg)) * (double)vd);",
                             "long hw = (long)(tan(half_fov_rad(p->fov_x_deg)) * (double)vd);"),
    "origin_rounds_up": ("o[k] = (int32_t)c - p->n[k] / 2;", "o[k] = (int32_t)c - (p->n[k] + 1) / 2;"),
    "start_voxel_skipped": ("if (in_grid(n, i[0], i[1], i[2])) {",
                            "if (in_grid(n, i[0], i[1], i[2]) && (i[0] != (int32_t)floorf(S[0]) || "
                            "i[1] != (int32_t)floorf(S[1]) || i[2] != (int32_t)floorf(S[2]))) {"),
    "fy_uses_fx": ("xyz[1] = ((float)v - K[3]) * d / K[1];", "xyz[1] = ((float)v - K[3]) * d / K[0];"),
    # the literal readings
    "skip_start_ignored_by_rays": ("dda_walk(p->n, S, D, (p->literal & OR_LIT_SKIP_START) != 0, ray_visit, &R)",
                                   "dda_walk(p->n, S, D, 0, ray_visit, &R)"),
    "skip_start_skips_two": ("        first = 0;\n", "        first = (first == 1) ? 2 : 0;\n"),
    "after_trace_tests_inflated": ("if (p->literal & OR_LIT_INFLATE_AFTER_TRACE) tested = occ_raw;",
                                   "if (p->literal & OR_LIT_INFLATE_AFTER_TRACE) tested = occ_inf;"),
    "loc_reading_tests_measurement": ("            tested = ms;\n", "            tested = occ_inf;\n"),
    "loc_reading_keeps_occupied": ("const int rays_last = (literal & OR_LIT_LOC_OCCUPANCY) != 0;",
                                   "const int rays_last = 0;"),
}

RUNNER = r"""
import json, sys
sys.path[:0] = [%(tests)r, %(root)r]
from oracle.oracle import Oracle
import oracle_pins
orc = Oracle(%(lib)r)
failed = []
for chk in oracle_pins.ALL_CHECKS:
    try:
        chk(orc)
    except AssertionError:
        failed.append(chk.__name__)
print(json.dumps(failed))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    from oracle import build as obuild
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found exactly once: " + name
    d = tmp_path / "src"
    d.mkdir()
    (d / "vg_oracle.c").write_text(src.replace(old, new))
    (d / "vg_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "vg_oracle.h")).read())
    lib = obuild.build(src=str(d / "vg_oracle.c"), out=str(tmp_path / "libmut.so"), force=True,
                       extra_flags=["-Wno-error"])
    code = RUNNER % {"tests": HERE, "root": ROOT, "lib": lib}
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    # the child must finish: a mutant that crashes the checks is a test bug
    assert res.returncode == 0, res.stderr[-2000:]
    failed = json.loads(res.stdout.strip().splitlines()[-1])
    print(name, "caught by", failed)
    assert failed, "mutant %s passed every pin" % name
