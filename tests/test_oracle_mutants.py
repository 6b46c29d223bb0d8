"""The oracle's pins must catch plausible mistakes.

Each mutant below is a one-line textual change to a temporary copy of
oracle/ec_oracle.c (a flipped comparison, a dropped term, a wrong sign or
index), compiled on the CPU and loaded as a separate module.  Every mutant must
fail at least one of the pin tests; the real oracle passes them all.
"""
import importlib.util
import os
import shutil
import subprocess
import sys
import types

import numpy as np
import pytest

import test_oracle_alpha as TA
import test_oracle_depth as TD
import test_oracle_depth_grad as TG
import test_oracle_rle as TR
import test_oracle_roi as TO
import test_oracle_assemble as TS
import test_oracle_schedules as TSC
import test_oracle_rle0 as TR0
import test_oracle_yuv as TY

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

MUTANTS = {
    "depth_tie_le": ("if (d < best_d[p])", "if (d <= best_d[p])"),
    "depth_background": ("best_d[p] = 1.0f; best_i[p] = -1;", "best_d[p] = 2.0f; best_i[p] = -1;"),
    "roi_inclusive_edge": ("(int64_t)px < (int64_t)r.x + r.w", "(int64_t)px <= (int64_t)r.x + r.w"),
    "merge_roi_drops_y": ("if (c.y < y0) y0 = c.y;", ""),
    "over_drops_T": ("C[ch] += T * c[ch];", "C[ch] += c[ch];"),
    "over_wrong_channel": ("T *= 1.0 - c[3];", "T *= 1.0 - c[2];"),
    "half_exponent": ("ldexp((double)(m + 1024), e - 25)", "ldexp((double)(m + 1024), e - 24)"),
    "grad_alpha_sign": ("d[3] = T[k] * (gp[3] - R);", "d[3] = T[k] * (gp[3] + R);"),
    "grad_R_no_transmit": ("R = gc + (1.0 - ck[3]) * R;", "R = gc + R;"),
    "grad_colour_T_next": ("d[0] = gp[0] * T[k];", "d[0] = gp[0] * T[k + 1];"),
    "depth_grad_to_all": ("d[ch] = winner[p] == i ? g[4 * p + ch] : 0.0f;", "d[ch] = g[4 * p + ch];"),
    "rle_repeat_threshold": ("if (L >= 3) {", "if (L >= 2) {"),
    "rle_repeat_control": ("out[o++] = (uint8_t)(128 + piece - 1);\n                out[o++] = b[i];",
                           "out[o++] = (uint8_t)(128 + piece);\n                out[o++] = b[i];"),
    "rle_piece_127": ("size_t piece = left >= 128 ? 128 : left;\n                out[o++] = (uint8_t)(128 + piece - 1);\n                out[o++] = b[i];",
                      "size_t piece = left >= 127 ? 127 : left;\n                out[o++] = (uint8_t)(128 + piece - 1);\n                out[o++] = b[i];"),
    "rle_literal_control": ("out[o++] = (uint8_t)(piece - 1);\n                memcpy(out + o, b + start + done, piece);",
                            "out[o++] = (uint8_t)(piece);\n                memcpy(out + o, b + start + done, piece);"),
    "swizzle_component_order": ("s |= ((b >> (6 - 2 * k)) & 3u) << (6 - 2 * j);",
                                "s |= ((b >> (6 - 2 * k)) & 3u) << (2 * j);"),
    "decoder_no_length_check": ("if (o != len) return ORC_ECORRUPT;", ""),
    "roi_depth_le": ("if (depth) return depth[e] < 1.0f;", "if (depth) return depth[e] <= 1.0f;"),
    "roi_half_sign": ("return (h[0] & 0x7FFFu) || (h[1] & 0x7FFFu)", "return (h[0] & 0xFFFFu) || (h[1] & 0x7FFFu)"),
    "roi_max_x_dropped": ("if (x > bx1) bx1 = x;", ""),
    "roi_occ_transposed": ("occ[(y / tile) * gw + x / tile] = 1;", "occ[(x / tile) * gw + y / tile] = 1;"),
    "roi_search_not_clipped": ("if (x1 > pvp.w) x1 = pvp.w;", ""),
    "tiles_ignore_roi": ("if (!in_rect(s->roi, px, py) || !in_rect(s->pvp, px, py)) continue;\n                const size_t e = (size_t)((py - s->pvp.y) * s->pitch + (px - s->pvp.x));\n                const size_t d",
                         "if (!in_rect(s->pvp, px, py)) continue;\n                const size_t e = (size_t)((py - s->pvp.y) * s->pitch + (px - s->pvp.x));\n                const size_t d"),
    "pixels_drop_offset": ("const int64_t dx = kx[k] + i * nx, dy = ky[k] + j * ny;", "const int64_t dx = i * nx, dy = ky[k] + j * ny;"),
    "average_no_rounding": ("((isum[ch] + (uint64_t)count / 2) / (uint64_t)count)", "((isum[ch]) / (uint64_t)count)"),
    "average_counts_all": ("                ++count;\n", ""),
    "rle0_literal_control": ("                out[o++] = (uint8_t)(piece - 1);\n                for (size_t k = 0; k < piece; ++k) {",
                             "                out[o++] = (uint8_t)(piece);\n                for (size_t k = 0; k < piece; ++k) {"),
    "rle0_tail_dropped": ("    if (len & 1) {\n        put_u32(out + o, e[len - 1]);\n        o += 4;\n    }\n", ""),
    "rle0_unit_halves_swapped": ("                put_u32(out + o, e[2 * i]);\n                put_u32(out + o + 4, e[2 * i + 1]);",
                                 "                put_u32(out + o, e[2 * i + 1]);\n                put_u32(out + o + 4, e[2 * i]);"),
    "yuv_luma_no_rounding": ("floor_div256(77 * R + 150 * G + 29 * B + 128)", "floor_div256(77 * R + 150 * G + 29 * B)"),
    "yuv_chroma_swapped": ("(uint32_t)((su + cnt / 2) / cnt) |\n                                               ((uint32_t)((sv + cnt / 2) / cnt) << 8)",
                           "(uint32_t)((sv + cnt / 2) / cnt) |\n                                               ((uint32_t)((su + cnt / 2) / cnt) << 8)"),
    "yuv_average_over_four": ("((uint32_t)((sa + cnt / 2) / cnt) << 16)", "((uint32_t)((sa + 2) / 4) << 16)"),
    "yuv_inverse_green_sign": ("clamp255(Y - floor_div256(88 * U + 183 * V + 128))", "clamp255(Y + floor_div256(88 * U + 183 * V + 128))"),
}


def _load_mutant(tmp_path, name, old, new):
    src = open(os.path.join(ORACLE, "ec_oracle.c")).read()
    assert src.count(old) == 1, f"mutant {name}: pattern must occur exactly once"
    d = tmp_path / name
    d.mkdir()
    shutil.copy(os.path.join(ORACLE, "ec_oracle.h"), d / "ec_oracle.h")
    (d / "ec_oracle.c").write_text(src.replace(old, new))
    so = d / "liboracle.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", str(so),
                           str(d / "ec_oracle.c"), "-lm"])
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}",
                                                  os.path.join(ORACLE, "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    mod._LIB = str(so)
    mod.build = lambda force=False: str(so)
    return mod


def _pins(orc):
    """The pin checks, as callables of the oracle module."""
    yield lambda: [TD.test_matches_independent_argmin(orc, s) for s in range(24)]
    yield lambda: TD.test_out_roi_is_bbox_union(orc)
    yield lambda: TD.test_single_source_is_masked_copy(orc)
    yield lambda: [TA.test_equal_alpha_closed_form(orc, n, a) for n, a in [(3, 0.1), (8, 0.3)]]
    yield lambda: TA.test_fp16_layers_decoded_exactly(orc)
    yield lambda: TA.test_roi_outside_is_transparent(orc)
    yield lambda: [TA.test_gradient_matches_exact_central_differences(orc, s) for s in range(3)]
    yield lambda: TA.test_gradient_closed_forms(orc)
    yield lambda: TG.test_depth_grad_routes_to_winner(orc)
    yield lambda: [TR.test_golden_worked_examples(orc, c) for c in range(len(TR._golden()))]
    yield lambda: TR.test_swizzle_is_a_bit_permutation(orc)
    yield lambda: [TR.test_streams_decode_and_have_canonical_size(orc, n, 1)
                   for n in ("run_lengths", "lit_run_mix", "boxes")]
    yield lambda: TR.test_decoder_rejects_corrupt_streams(orc)
    yield lambda: [TO.test_matches_numpy_reductions(orc, f, s) for f in ("depth", 0, 1, 2) for s in range(4)]
    yield lambda: TO.test_search_region_limits_the_scan(orc)
    yield lambda: TO.test_special_values(orc)
    yield lambda: TS.test_tile_order_roi_and_untouched_pixels(orc)
    yield lambda: [TS.test_pixel_decomposition_reassembles(orc, "rgba8", k) for k in ((2, 2), (4, 3))]
    yield lambda: TS.test_rgba8_average_rounding_and_coverage(orc)
    yield lambda: TS.test_float_average_matches_numpy_mean(orc, "f32", 1)
    yield lambda: [TR0.test_streams_decode_and_have_canonical_size(orc, n)
                   for n in ("unit_run_lengths", "straddle_odd", "boxes", "pairs_of_pixels")]
    yield lambda: TR0.test_incompressible_meets_its_bound(orc)
    yield lambda: [TY.test_luma_and_chroma_follow_the_float_transform(orc, h, w) for h, w in ((8, 8), (5, 7))]
    yield lambda: TY.test_grey_round_trips_exactly(orc)
    yield lambda: TY.test_uniform_blocks_round_trip_within_bound(orc)


def _caught(orc):
    for pin in _pins(orc):
        try:
            pin()
        except (AssertionError, RuntimeError, ValueError, IndexError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    mut = _load_mutant(tmp_path, name, old, new)
    assert _caught(mut), f"mutant {name} survived every pin"


def test_real_oracle_passes_all_pins(orc):
    assert not _caught(orc)


# ---- schedule planner and executor (oracle/schedules.py, Python) ----------

SCHED_MUTANTS = {
    "sched_units_reversed": ("            for u in group:\n                for m in u:\n                    p = intersect",
                             "            for u in reversed(group):\n                for m in u:\n                    p = intersect"),
    "sched_chain_front_back": ("[[[l], [l + 1]]]", "[[[l + 1], [l]]]"),
    "sched_bands_ceil": ("a, b = y + (j * h) // k, y + ((j + 1) * h) // k",
                         "a, b = y + (j * h) // k, y + ((j + 1) * h + k - 1) // k"),
    "sched_self_messages": ("if m != r:\n                        lv.messages.append",
                            "if True:\n                        lv.messages.append"),
    "sched_intersect_short": ("x1, y1 = min(a[0] + a[2], b[0] + b[2]), min(",
                              "x1, y1 = min(a[0] + a[2], b[0] + b[2]) - 1, min("),
    "sched_halves_overlap": ("return (x, y, w, m), (x, y + m, w, h - m)", "return (x, y, w, m + 1), (x, y + m, w, h - m)"),
}


def _load_sched_mutant(name, old, new):
    src = open(os.path.join(ORACLE, "schedules.py")).read()
    assert src.count(old) == 1, f"mutant {name}: pattern must occur exactly once"
    mod = types.ModuleType(f"oracle._sched_mutant_{name}")
    mod.__package__ = "oracle"
    sys.modules[mod.__name__] = mod
    exec(compile(src.replace(old, new), f"schedules_{name}.py", "exec"), mod.__dict__)
    return mod


def _sched_caught(mod, monkeypatch):
    monkeypatch.setattr(TSC, "S", mod)
    pins = [
        lambda: [TSC.test_schedule_equals_single_pass(a, True) for a in TSC.ALGOS],
        lambda: [TSC.test_final_regions_partition_the_frame(a) for a in TSC.ALGOS],
        lambda: [TSC.test_full_frame_transfers(a, c) for a, c in TSC.FULL_FRAME_COUNTS],
        lambda: TSC.test_two_three_swap_of_three_is_direct_send(),
        lambda: TSC.test_direct_send_moves_only_roi_pixels(),
    ]
    for pin in pins:
        try:
            pin()
        except (AssertionError, RuntimeError, ValueError, IndexError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(SCHED_MUTANTS))
def test_schedule_pins_catch_mutant(name, monkeypatch):
    mod = _load_sched_mutant(name, *SCHED_MUTANTS[name])
    assert _sched_caught(mod, monkeypatch), f"mutant {name} survived every schedule pin"


def test_real_schedule_oracle_passes_all_pins(monkeypatch):
    from oracle import schedules
    assert not _sched_caught(schedules, monkeypatch)
