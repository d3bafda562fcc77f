"""Planted mistakes in the oracle, on the CPU: every mutant of oracle.c below
(one plausible slip each: a dropped term, a wrong sign, index or word, a
transposed operand, an off-by-one) must fail at least one of the oracle's pins
(tests/test_oracle_pins.py, tests/test_oracle_mlp.py).  The mutants are built
from a copy of the source in a temporary directory; oracle.c is not touched.
An unmutated build of the same copy passes the pins, so a failure comes from
the planted mistake and not from the harness."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_mlp.py"]

# (name, passage the mistake breaks, original text, mutated text)
MUTANTS = [
    # Section 2.1: the image K_i
    ("image_drops_sign", "Sec. 2.1",
     "K[net->dst[e]] += (s[net->src[e]] / t[e]) * w[e] * p[e];",
     "K[net->dst[e]] += (s[net->src[e]] / t[e]) * w[e];"),
    ("image_transposed_edge", "Sec. 2.1",
     "K[net->dst[e]] += (s[net->src[e]] / t[e]) * w[e] * p[e];",
     "K[net->src[e]] += (s[net->dst[e]] / t[e]) * w[e] * p[e];"),
    ("image_threshold_as_compare", "Sec. 2.1",
     "K[net->dst[e]] += (s[net->src[e]] / t[e]) * w[e] * p[e];",
     "K[net->dst[e]] += (s[net->src[e]] >= t[e]) * w[e] * p[e];"),
    ("target_upper_clamp_1", "Sec. 2.1",
     "int32_t tgt = K[i] < 0 ? 0 : (K[i] > 2 ? 2 : K[i]);",
     "int32_t tgt = K[i] < 0 ? 0 : (K[i] > 1 ? 1 : K[i]);"),
    # Section 2.2: memory, priority, move
    ("memory_off_by_one", "Sec. 2.2, m",
     "if (cnt[i] >= m[i] + 1 && selected) {",
     "if (cnt[i] >= m[i] && selected) {"),
    ("memory_ignores_direction", "Sec. 2.2, m",
     "cnt[i] = (drv == dir[i]) ? cnt[i] + 1 : 1;",
     "cnt[i] = cnt[i] + 1;"),
    ("priority_ignores_last_update", "Sec. 2.2, u",
     "prio[i] = (net->sync || net->async_sel) ? 1 : u[i] * (tau - last[i]);",
     "prio[i] = (net->sync || net->async_sel) ? 1 : u[i] * tau;"),
    ("priority_ignores_speed", "Sec. 2.2, u",
     "prio[i] = (net->sync || net->async_sel) ? 1 : u[i] * (tau - last[i]);",
     "prio[i] = (net->sync || net->async_sel) ? 1 : (tau - last[i]);"),
    ("move_ignores_distance", "Sec. 2.2, d",
     "move[i] = drv * (d[i] < mag ? d[i] : mag);",
     "move[i] = drv * d[i];"),
    ("last_update_not_recorded", "Sec. 2.2",
     "                    last[i] = tau;\n",
     ""),
    ("only_first_tied_node_moves", "Sec. 2.2",
     "                    s[i] += move[i];\n",
     "                    s[i] += move[i];\n                    pmax = -1;\n"),
    ("memory_kept_after_move", "Sec. 2.2, m",
     "                    last[i] = tau;\n                    cnt[i] = 0;\n                    dir[i] = 0;\n",
     "                    last[i] = tau;\n"),
    ("synchronous_scheme_ignored", "Sec. 2.2, synchronous updating",
     "prio[i] = (net->sync || net->async_sel) ? 1 : u[i] * (tau - last[i]);",
     "prio[i] = net->async_sel ? 1 : u[i] * (tau - last[i]);"),
    ("asynchronous_selection_shifted", "Sec. 2.2, asynchronous updating",
     "net->async_sel[(size_t)c * net->n_times_sel + tau] == i;",
     "net->async_sel[(size_t)c * net->n_times_sel + tau - 1] == i;"),
    # Section 2.3: weights and objective
    ("weight_drops_one", "Sec. 2.3",
     "W[k] = (uint8_t)((G < 0 ? -G : G) + 1);",
     "W[k] = (uint8_t)(G < 0 ? -G : G);"),
    ("gradient_ignores_observation", "Sec. 2.3",
     "if (tau > 0 && tc->observed[k - N]) G =",
     "if (tau > 0) G ="),
    ("gradient_wrong_neighbour", "Sec. 2.3",
     "(int32_t)tc->ref[k] - (int32_t)tc->ref[k - N];",
     "(int32_t)tc->ref[k] - (int32_t)tc->ref[k - 1];"),
    ("score_drops_abs", "Sec. 2.3",
     "y += (int64_t)W[k] * (e < 0 ? -e : e);",
     "y += (int64_t)W[k] * e;"),
    ("unobserved_entries_weighted", "Sec. 2.3",
     "if (!tc->observed[k]) { W[k] = 0; continue; }",
     "if (!tc->observed[k]) { W[k] = 1; continue; }"),
    # Table 1 and Section 2.5.3: GetCandidate
    ("alternatives_include_current", "Table 1, GetCandidate",
     "        if (vals[k] == x[j]) continue;\n        y[j] = vals[k];",
     "        y[j] = vals[k];"),
    ("proposal_ignores_constraints", "Sec. 2.5.3",
     "if (constraints_hold(net, y)) alts[n_alt++] = vals[k];",
     "alts[n_alt++] = vals[k];"),
    ("value_drawn_from_index_word", "Table 1, GetCandidate",
     "*v_out = alts[pick(r1, (uint32_t)n_alt)];",
     "*v_out = alts[pick(r0, (uint32_t)n_alt)];"),
    ("constraint_ignores_sign", "Sec. 2.5.3",
     "if (net->dst[e] == i && x[e] != 0 && x[E + e] == 1) pos_in++;",
     "if (net->dst[e] == i && x[e] != 0) pos_in++;"),
    # Table 1: acceptance, levels, best vectors
    ("threshold_multiplies_temperature", "Table 1, A = exp(-dE / T)",
     "double a = exp(-(double)dE / T) * 4294967296.0;",
     "double a = exp(-(double)dE * T) * 4294967296.0;"),
    ("acceptance_uses_index_word", "Table 1",
     "int accept = dE <= 0 || r[2] < orc_threshold(T, dE);",
     "int accept = dE <= 0 || r[0] < orc_threshold(T, dE);"),
    ("level_count_off_by_one", "Table 1, while T > T_min",
     "    while (T > T_min) {\n        n++;",
     "    while (T >= T_min * rho) {\n        n++;"),
    ("reset_at_level_end", "Table 1",
     "if (sched->reset_to_best && g % n_iter == 0) {",
     "if (sched->reset_to_best && (g + 1) % n_iter == 0) {"),
    ("uphill_counts_neutral_moves", "Table 1",
     "if (dE > 0) st->n_uphill[k]++;",
     "if (dE >= 0) st->n_uphill[k]++;"),
    ("null_moves_not_counted", "Table 1",
     "                st->n_null[k]++;\n",
     ""),
    ("argmin_last_on_ties", "Table 1, global argmin",
     "if (st->d_best[k] < st->d_best[b]) b = k;",
     "if (st->d_best[k] <= st->d_best[b]) b = k;"),
    ("groups_ignored", "Sec. 4.5, grouped reduction",
     "const int32_t end = first + G < n_chains ? first + G : n_chains;",
     "const int32_t end = n_chains;"),
    # the generator and the initial vectors
    ("philox_key_constant", "Philox4x32-10 (Salmon et al.)",
     "k1 += 0xBB67AE85u;",
     "k1 += 0x9E3779B9u;"),
    ("philox_crossed_halves", "Philox4x32-10 (Salmon et al.)",
     "c0 = hi1 ^ c1 ^ k0;",
     "c0 = hi0 ^ c1 ^ k0;"),
    ("init_same_word_for_every_parameter", "Sec. 2.4.2",
     "x[j] = vals[pick(r[j & 3], (uint32_t)n)];",
     "x[j] = vals[pick(r[0], (uint32_t)n)];"),
    ("init_repair_wrong_sign", "Sec. 2.5.3",
     "if (!is_frozen(net, E + e)) x[E + e] = 1;",
     "if (!is_frozen(net, E + e)) x[E + e] = -1;"),
    ("asynchronous_scheme_proposes_speeds", "Sec. 2.2, asynchronous updating",
     "return !((net->sync || net->async_sel) && kind_of(net, j, &idx) == K_U);",
     "return !(net->sync && kind_of(net, j, &idx) == K_U);"),
    ("out_edge_constraint_ignores_weight", "Sec. 2.5.3",
     "if (net->src[e] == i && x[e] != 0) out_nz++;",
     "if (net->src[e] == i) out_nz++;"),
    ("conditions_share_one_trajectory", "Sec. 2.3, S per condition",
     "int32_t rc = orc_simulate(net, tc, x, c, buf + (size_t)c * T * N);",
     "int32_t rc = orc_simulate(net, tc, x, c, buf);"),
    ("row_t0_not_recorded", "Sec. 2.3, S row t0",
     "        S[i] = (uint8_t)s[i];\n",
     ""),
    ("pick_by_modulo", "Table 1, a uniform draw",
     "return (uint32_t)(((uint64_t)r * n) >> 32); }",
     "return r % n; }"),
    ("proposal_index_off_by_one", "Table 1, GetCandidate",
     "        if (seen++ == want) { j = k; break; }",
     "        if (++seen == want) { j = k; break; }"),
    ("threshold_without_cap", "Table 1, A = exp(-dE / T)",
     "    if (f >= 4294967295.0) return 0xFFFFFFFFu;\n",
     ""),
    ("level_temperature_one_level_late", "Table 1, T <- rho T",
     "for (int64_t l = 0; l < level; l++) T *= alpha;",
     "for (int64_t l = 0; l <= level; l++) T *= alpha;"),
    ("repair_weight_from_index_word", "Sec. 2.5.3",
     "            x[e] = (int8_t)(1 + (r[1] & 1u));\n            break;",
     "            x[e] = (int8_t)(1 + (r[0] & 1u));\n            break;"),
    ("knockout_not_zero_at_t0", "Sec. 2.4, knockouts",
     "s[i] = (ko && ko[i]) ? 0 : tc->init[(size_t)c * N + i];",
     "s[i] = tc->init[(size_t)c * N + i];"),
    ("knockout_node_updates", "Sec. 2.4, knockouts",
     "            if (ko && ko[i]) continue;\n",
     ""),
    # the screening MLP
    ("mlp_drops_second_bias", "screen: a2 = b2 + W2^T h1",
     "            double s = b2[k];",
     "            double s = 0.0;"),
    ("mlp_bias_gradient_without_relu_mask", "screen: dL/db1",
     "            d1[i] = a1[i] > 0.0 ? s : 0.0;",
     "            d1[i] = s;"),
    ("mlp_output_bias_gradient_dropped", "screen: dL/db3",
     "        if (gb3) *gb3 += dy;",
     "        if (gb3) *gb3 += 0.0;"),
    ("mlp_first_gradient_overwritten", "screen: dL/dW1 sums over the batch",
     "for (int32_t i = 0; i < H1; i++) gW1[(size_t)r * H1 + i] += d1[i];",
     "for (int32_t i = 0; i < H1; i++) gW1[(size_t)r * H1 + i] = d1[i];"),
    ("mlp_loss_absolute", "screen: mean (y - t)^2",
     "if (loss) *loss += diff * diff / B;",
     "if (loss) *loss += fabs(diff) / B;"),
    ("mlp_output_gradient_without_relu", "screen: dL/dw3 = dy h2",
     "if (gw3) gw3[k] += dy * h2;",
     "if (gw3) gw3[k] += dy * a2[k];"),
    ("mlp_drops_hidden_relu", "screen: h1 = relu(a1)",
     "s += (a1[i] > 0.0 ? a1[i] : 0.0) * W2[(size_t)i * H2 + k];",
     "s += a1[i] * W2[(size_t)i * H2 + k];"),
    ("mlp_gradient_transposed", "screen: dL/dW2",
     "if (gW2) gW2[(size_t)i * H2 + k] += h1 * d2[k];",
     "if (gW2) gW2[(size_t)k * H1 + i] += h1 * d2[k];"),
    ("mlp_loss_gradient_halved", "screen: d(mean (y - t)^2)/dy",
     "const double dy = 2.0 * diff / B;",
     "const double dy = diff / B;"),
    ("mlp_onehot_reversed", "screen: one-hot of x",
     "if (vals[k] == v) return off[j] + k;",
     "if (vals[k] == v) return off[j] + n - 1 - k;"),
]


def _build(tmp, name, text):
    src = tmp / f"{name}.c"
    src.write_text(text)
    lib = tmp / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-w",
                           "-I", os.path.join(ROOT, "oracle"), "-o", str(lib), str(src), "-lm"])
    return lib


def _run_pins(lib):
    env = dict(os.environ, ORC_LIB=str(lib))
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q",
                            "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=240)
    except subprocess.TimeoutExpired:
        return None
    return r.returncode


def test_mutant_table_matches_the_source():
    text = open(SRC).read()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, _, orig, mut in MUTANTS:
        assert text.count(orig) == 1, f"{name}: the original text must occur exactly once"
        assert orig != mut


def test_every_planted_mistake_fails_a_pin(tmp_path):
    text = open(SRC).read()
    libs = {"unmutated": _build(tmp_path, "unmutated", text)}
    for name, _, orig, mut in MUTANTS:
        libs[name] = _build(tmp_path, name, text.replace(orig, mut))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        rc = dict(zip(libs, ex.map(_run_pins, libs.values())))
    assert rc.pop("unmutated") == 0, "the pins must pass on an unmutated build of the copy"
    survivors = [name for name, code in rc.items() if code == 0]
    assert not survivors, f"planted mistakes no pin detects: {survivors}"
