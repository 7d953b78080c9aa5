"""The oracle's pins catch plausible mistakes: each case below plants one mistake in a
copy of oracle/atsfft_oracle.c (a flipped sign, a swapped index, a dropped term, an
off-by-one), builds it with gcc and runs tests/test_oracle_pins.py against that build;
at least one pin must fail.  The unchanged copy must pass them all (the control case),
so a failure is the mistake's doing.  CPU only; the planted mistakes live in temporary
copies and never touch the oracle itself."""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "atsfft_oracle.c")
HDR = os.path.join(ROOT, "oracle", "atsfft_oracle.h")
PINS = os.path.join(HERE, "test_oracle_pins.py")

# name -> (text in the oracle, replacement, the step of the paper it breaks)
MUTANTS = {
    "estimate_phase_sign": (
        "double ang = -2.0 * M_PI * (double)m / (double)n; /* omega^{tau i} */",
        "double ang = 2.0 * M_PI * (double)m / (double)n; /* omega^{tau i} */",
        "Eq. (11): the phase omega^{tau i}"),
    "estimate_gain_multiplied": (
        "est[s * L + l] = Z[bucket] * ph / gain;",
        "est[s * L + l] = Z[bucket] * ph * gain;",
        "Eq. (11): division by the window gain"),
    "reverse_hash_sigma_not_inverse": (
        "votes[mulmod(si1, pp, n)]++;",
        "votes[mulmod(hp[0], pp, n)]++;",
        "Section II-B: reverse hash through sigma^{-1}"),
    "median_index": (
        "return re[L / 2] + I * im[L / 2];",
        "return re[L / 2 - 1] + I * im[L / 2 - 1];",
        "Section II-B: median of the L estimates"),
    "bins_2d_transposed": (
        "Z[b1 * B + b2] += g1",
        "Z[b2 * B + b1] += g1",
        "Eq. (2) / Lemma 2 in 2D: bucket (b1, b2) row-major"),
    "half_bin_modulation_sign": (
        "double ang = M_PI * (double)t / (double)n;",
        "double ang = -M_PI * (double)t / (double)n;",
        "flat window of Section II-A-2: pass band centred on the bucket"),
    "gaussian_width": (
        "double ss = (double)B * q / (M_PI * alpha);",
        "double ss = (double)B * q / (2.0 * M_PI * alpha);",
        "Eq. (9): Gaussian width of the flat window"),
    "response_offset_grid": (
        "int64_t o2 = 2 * j - D + 1; /* 2*o, an odd integer */",
        "int64_t o2 = 2 * j - D; /* 2*o, an odd integer */",
        "Eq. (11): window gain at the half-integer offset"),
    "vote_threshold": (
        "int need = (p->loops_loc + 1) / 2;",
        "int need = p->loops_loc / 2;",
        "Section II-B: votes in at least half of the location loops"),
    "tie_direction": (
        "return d1 < 0 || (d1 == 0 && d2 < 0);",
        "return d1 > 0 || (d1 == 0 && d2 > 0);",
        "Section III-A local maxima: ties go to the later bucket"),
    "neighbourhood_2d_four": (
        "if (d1 == 0 && d2 == 0) continue;",
        "if ((d1 == 0 && d2 == 0) || (d1 != 0 && d2 != 0)) continue;",
        "Section III-A / Fig. 5: eight neighbours in 2D"),
    "threshold_median_term_dropped": (
        "return fmax(thr_rel * mx, thr_med * med);",
        "return thr_rel * mx;",
        "Section III-A: threshold against the median"),
    "bucket_floor_not_round": (
        "int64_t q = (2 * p + 1 + D) / (2 * D);",
        "int64_t q = (2 * p + 1) / (2 * D);",
        "Eq. (10): bucket of a coordinate by rounding"),
    "controller_stop_delta1": (
        "if (trial > 0 && r < p->delta2) break;",
        "if (trial > 0 && r < p->delta1) break;",
        "Eqs. (12)-(14): stop below delta2"),
    "top_num_pivot_off_by_one": (
        "double V = v[num - 1].e,",
        "double V = v[num].e,",
        "Algorithm 1 'find num largest': the num-th largest"),
    "fft_twiddle_sign": (
        "double ang = -2.0 * M_PI * (double)j / (double)m;",
        "double ang = 2.0 * M_PI * (double)j / (double)m;",
        "the B-point DFT's sign convention"),
    "inverse_mod_too_few_steps": (
        "for (int it = 0; it < 6; it++) x = x * (2 - s * x);",
        "for (int it = 0; it < 2; it++) x = x * (2 - s * x);",
        "Def. 1: sigma^{-1} mod n"),
    "estimate_with_location_hashes": (
        "orc_hash_params(cx->seed, cx->p->est_reuse_loc ? 1 : 2, l, n, ndim, hp);",
        "orc_hash_params(cx->seed, 1, l, n, ndim, hp);",
        "Eq. (11): the estimation hash's own permutation"),
    "reverse_hash_no_half_bucket_shift": (
        "int64_t pp = emod(c * D - D / 2 + q, n);",
        "int64_t pp = emod(c * D + q, n);",
        "Section II-B: preimage of a bucket centred at c D - 1/2"),
    "reverse_hash_2d_no_half_bucket_shift": (
        "int64_t i = mulmod(si1, emod(c1 * D - D / 2 + q1, n), n);",
        "int64_t i = mulmod(si1, emod(c1 * D + q1, n), n);",
        "Section II-B in 2D: preimage rows of a bucket"),
    "window_normalisation": (
        "double A = (double)n / sum;",
        "double A = 1.0 / sum;",
        "Section II-A-2: window normalised to unit gain"),
    "response_scale": (
        "resp[j] = acc / (double)n;",
        "resp[j] = acc;",
        "Eq. (11): window gain Ghat'"),
    "default_thr_med": (
        "p->thr_med = 20.0;",
        "p->thr_med = 10.0;",
        "Section III-A: the median factor of the threshold"),
    "default_thr_rel": (
        "p->thr_rel = 1e-3;",
        "p->thr_rel = 1e-2;",
        "Section III-A: the relative factor of the threshold"),
    "default_delta2": (
        "p->delta2 = 0.05;",
        "p->delta2 = 0.04;",
        "Eq. (14): delta2 = 5 %"),
    "default_tie_band": (
        "p->tie_eta = 1e-2;",
        "p->tie_eta = 0.0;",
        "Section III-A local maxima: the tie band"),
    "sigma_not_forced_odd": (
        "out[2 * d + 0] = (int64_t)((orc_splitmix64_next(&st) & mask) | 1);",
        "out[2 * d + 0] = (int64_t)(orc_splitmix64_next(&st) & mask);",
        "Def. 1: sigma invertible mod n"),
    "estimate_2d_phase_sign": (
        "m = (m + mulmod(hp[3], j, n)) % n;",
        "m = emod(m - mulmod(hp[3], j, n), n);",
        "Eq. (11) in 2D: omega^{tau1 i + tau2 j}"),
    "neighbour_before_skipped": (
        "for (int d2 = -1; d2 <= 1; d2++) {",
        "for (int d2 = 0; d2 <= 1; d2++) {",
        "Section III-A: both neighbours of a local maximum"),
    "tuning_previous_count_kept": (
        "k_prev = k_cur;",
        "(void)k_prev;",
        "Eq. (12): r against the previous trial's count"),
    "half_bin_missing_second_axis": (
        "(w->taps[t2 + w->h] * half_bin(t2, N))",
        "(w->taps[t2 + w->h])",
        "flat window in 2D: half-bin modulation on both axes"),
    "location_loop_dropped": (
        "for (int l = 0; l < p->loops_loc; l++) {",
        "for (int l = 0; l < p->loops_loc - 1; l++) {",
        "Section II-B: votes over all L_loc location hashes"),
    "fixed_k_bucket_rule_1d": (
        "int bf = ndim == 1 ? (m + 1) / 2 : (m + 3) / 4;",
        "int bf = ndim == 1 ? m / 2 : (m + 3) / 4;",
        "fixed-k mode: the smallest B with B^2 >= n k"),
    "fixed_k_bucket_rule_2d": (
        "int bf = ndim == 1 ? (m + 1) / 2 : (m + 3) / 4;",
        "int bf = ndim == 1 ? (m + 1) / 2 : (m + 1) / 4;",
        "fixed-k mode in 2D: the smallest B with B^4 >= N^2 k"),
    "reuse_estimates_from_fresh_hashes": (
        "hash_any(cx, B, p->est_reuse_loc ? 1 : 2, l, &w, Z);",
        "hash_any(cx, B, 2, l, &w, Z);",
        "estimation reusing the location hashes"),
    "k_hint_start": (
        "int want = ndim == 1 ? ilog2(2 * k_hint) : (ilog2(2 * k_hint) + 1) / 2;",
        "int want = ndim == 1 ? ilog2(k_hint) : (ilog2(2 * k_hint) + 1) / 2;",
        "Algorithm 2's initial B from a sparsity hint"),
    "capacity_status_off_by_one": (
        "if (count > capacity && status == ORC_OK) status = ORC_E_CAPACITY;",
        "if (count >= capacity && status == ORC_OK) status = ORC_E_CAPACITY;",
        "output capacity: an error only when the outputs do not fit"),
    "not_sparse_on_first_trial": (
        "if (trial > 0) status = ORC_E_NOT_SPARSE;",
        "status = ORC_E_NOT_SPARSE;",
        "Eq. (14): doubling past the largest B"),
    "trial_cap_off_by_one": (
        "if (trial + 1 >= p->tune_max) {",
        "if (trial >= p->tune_max) {",
        "Algorithm 2: at most tune_max trials"),
    "largest_b_default": (
        "int b_hi = p->b_max_log2 ? p->b_max_log2 : (ndim == 1 ? lgn - 4 : lgn - 2);",
        "int b_hi = p->b_max_log2 ? p->b_max_log2 : (ndim == 1 ? lgn - 3 : lgn - 2);",
        "the B range's upper end (bucket width >= 16 bins)"),
    "smallest_b_default_2d": (
        "int b_lo = p->b_min_log2 ? p->b_min_log2 : (ndim == 1 ? 4 : 3);",
        "int b_lo = p->b_min_log2 ? p->b_min_log2 : (ndim == 1 ? 4 : 4);",
        "Algorithm 2's smallest B in 2D"),
    "zero_signal_not_detected": (
        "if (maxE == 0.0) { /* nothing in the window: the signal is zero there */",
        "if (0) { /* nothing in the window: the signal is zero there */",
        "a zero signal gives an empty output"),
    "threshold_median_rank": (
        "double med = tmp[nb / 2], mx = tmp[nb - 1];",
        "double med = tmp[nb / 2 - 1], mx = tmp[nb - 1];",
        "Section III-A: the median of the energies"),
    "reverse_hash_2d_second_axis_sigma": (
        "int64_t si2 = ndim == 2 ? orc_inv_mod(hp[2], n) : 0;",
        "int64_t si2 = ndim == 2 ? hp[2] : 0;",
        "Section II-B in 2D: sigma_2^{-1} on the second axis"),
    "estimate_2d_second_axis_gain": (
        "gain *= resp[(o2 + D - 1) / 2];",
        "gain *= 1.0;",
        "Eq. (11) in 2D: the second axis's window gain"),
    "clamped_window_keeps_its_width": (
        "*s = (double)hmax / q;",
        "*s = ss;",
        "flat window clamped to the signal: the Gaussian narrowed to fit"),
    "tap_box_scale": (
        "double box = (t == 0) ? D : sin_pi_t_over_B(t, B) / (M_PI * (double)t / (double)n);",
        "double box = (t == 0) ? D : sin_pi_t_over_B(t, B) / (M_PI * (double)t / (double)B);",
        "Eq. (8): the box car's samples against its centre tap"),
    "permutation_tau_sign": (
        "int64_t a = (mulmod(sigma, emod(t, n), n) + tau) % n;",
        "int64_t a = emod(mulmod(sigma, emod(t, n), n) - tau, n);",
        "Def. 1: x at sigma t + tau"),
    "estimate_phase_uses_sigma": (
        "int64_t m = mulmod(hp[1], i, n);",
        "int64_t m = mulmod(hp[0], i, n);",
        "Eq. (11): the phase omega^{tau i}, tau not sigma"),
    "dominance_without_tie_band": (
        "if (Ec > (1.0 + eta) * Em) return 1;",
        "if (Ec > Em) return 1;",
        "Section III-A local maxima: energies within the band are tied"),
    "threshold_margin_skipped": (
        "            if (g < margin) margin = g;\n            log_decision(lg, ORC_DEC_THRESHOLD, c, -1, g);",
        "            log_decision(lg, ORC_DEC_THRESHOLD, c, -1, g);",
        "decision margins: the threshold test of Section III-A"),
    "threshold_decision_not_logged": (
        "            log_decision(lg, ORC_DEC_THRESHOLD, c, -1, g);",
        "            (void)0;",
        "near-decision log: the threshold test of Section III-A"),
    "dominance_margin_skipped": (
        "                if (g < margin) margin = g;\n                log_decision(lg, ORC_DEC_DOMINANCE",
        "                log_decision(lg, ORC_DEC_DOMINANCE",
        "decision margins: the tie band of Section III-A"),
    "dominance_gap_one_edge": (
        "double g = fmin(rel_gap(Ec, (1.0 + eta) * Em), rel_gap(Em, (1.0 + eta) * Ec));",
        "double g = rel_gap(Ec, (1.0 + eta) * Em);",
        "decision margins: both edges of the tie band"),
    "margin_mode_ignored": (
        "int changes = mode == 0 ? (before_c + before_m != after_c + after_m)",
        "int changes = 1 ? (before_c + before_m != after_c + after_m)",
        "decision margins: the location outcome is the maxima set, not their number"),
    "topnum_gap_one_edge": (
        "double g = fmin(rel_gap(e, hi), rel_gap(e, lo));",
        "double g = rel_gap(e, hi);",
        "decision margins: both edges of Algorithm 1's cutoff band"),
    "pivot_shifts_not_logged": (
        "if (!lg || nflip == 0 || !lg->rec || first + nflip > lg->cap) return ns;",
        "return ns;",
        "near-decision log: selections moved by a local-maximum flip"),
    "location_margin_not_kept": (
        "    if (marg < *margin) *margin = marg;",
        "    (void)marg;",
        "decision margins of the location hashes"),
    "tuning_margin_not_kept": (
        "        if (marg < res->min_margin) res->min_margin = marg;",
        "        (void)marg;",
        "decision margins of the tuning trials (Eqs. (12)-(14))"),
    "tap_envelope_width": (
        "double env = exp(-((double)t * (double)t) / (2.0 * s * s));",
        "double env = exp(-((double)t * (double)t) / (4.0 * s * s));",
        "Eq. (9): the Gaussian envelope of the taps"),
}


def _build(tmp_path, name):
    src = open(SRC).read()
    if name != "control":
        old, new, _ = MUTANTS[name]
        assert src.count(old) == 1, f"{name}: the text to mutate is not unique in the oracle"
        src = src.replace(old, new)
    work = tmp_path / name
    work.mkdir()
    (work / "atsfft_oracle.c").write_text(src)
    shutil.copy(HDR, work / "atsfft_oracle.h")
    so = work / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so),
                    str(work / "atsfft_oracle.c"), "-lm"], check=True)
    return str(so)


def _run_pins(so):
    env = dict(os.environ, ATSFFT_ORACLE_LIB=so, OMP_NUM_THREADS="1",
               OPENBLAS_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q",
                           "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


@pytest.fixture(scope="module")
def runs(tmp_path_factory):
    """Every build (the control and each mutant) against the pins, several at a time."""
    tmp = tmp_path_factory.mktemp("mutants")
    names = ["control"] + sorted(MUTANTS)
    libs = {nm: _build(tmp, nm) for nm in names}
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {nm: ex.submit(_run_pins, libs[nm]) for nm in names}
        return {nm: f.result() for nm, f in futs.items()}


def test_control_copy_passes_every_pin(runs):
    r = runs["control"]
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(runs, name):
    r = runs[name]
    # pytest exit code 1: some tests failed (anything else is a harness problem)
    assert r.returncode == 1, (f"{name} ({MUTANTS[name][2]}) survived the pins"
                               if r.returncode == 0 else r.stdout[-2000:] + r.stderr[-2000:])
