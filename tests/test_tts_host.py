"""Host logic of the time-to-solution search (no GPU): the Delta-t_max scan, the common-sample
error measure and the leap-frog stability step."""
import math

import numpy as np
import pytest

from paper_2401_16322_gb300.tts import (LEAPFROG_DIVISORS, SCAN_PLAN, Candidate, dt_max_scan,
                                        leapfrog_step, pml_beta0, rel_l2_common)


def test_scan_stops_at_the_largest_passing_step():
    errs = {6: float("inf"), 5: 3e-3, 4: 2e-4, 3: 9e-5, 2: 1e-6}
    k, seen = dt_max_scan([6, 5, 4, 3, 2], errs.__getitem__, 1e-4)
    assert k == 3
    assert [s[0] for s in seen] == [6, 5, 4, 3]


def test_scan_without_a_pass_evaluates_everything():
    k, seen = dt_max_scan([3, 2, 1], lambda k: 1.0, 1e-4)
    assert k is None and len(seen) == 3


def test_scan_treats_nan_as_failure():
    k, _ = dt_max_scan([2, 1], {2: float("nan"), 1: 0.0}.__getitem__, 1e-4)
    assert k == 1


def test_scan_orders_are_descending_steps():
    for _method, _ms, ks in SCAN_PLAN:
        assert list(ks) == sorted(ks, reverse=True)
    assert list(LEAPFROG_DIVISORS) == sorted(LEAPFROG_DIVISORS)


def test_common_sample_error_coarse_against_fine():
    # reference sampled at (s+1) dt_ref, candidate at (s+1) 3 dt_ref: samples 2, 5, 8, ... of ref
    ref = np.arange(1, 31, dtype=float)[:, None] * np.ones((1, 4))
    seis = ref[2::3].copy()
    assert rel_l2_common(seis, 3.0, ref, 1.0) == 0.0
    seis[0, 0] += 1.0
    b = ref[2::3]
    assert math.isclose(rel_l2_common(seis, 3.0, ref, 1.0), 1.0 / np.linalg.norm(b), rel_tol=1e-15)


def test_common_sample_error_fine_against_coarse():
    ref = np.arange(1, 11, dtype=float)[:, None]
    seis = np.repeat(ref, 4, axis=0)          # at dt_ref / 4: sample 4k+3 equals ref[k]
    assert rel_l2_common(seis, 0.25, ref, 1.0) == 0.0


def test_leapfrog_step_formula():
    # omega_max = c sqrt(2 |S2|) / dx with |S2| = 6.5016 (8th order): 2 / omega_max
    c, dx = 4500.0, 10.0
    w = c * math.sqrt(2 * 6.501587301587302) / dx
    assert math.isclose(leapfrog_step(c, dx), 2.0 / w, rel_tol=1e-15)
    # the 8th-order centred second-derivative symbol at the Nyquist frequency
    a = [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]
    s2 = a[0] + 2 * sum(a[k] * math.cos(k * math.pi) for k in range(1, 5))
    assert math.isclose(abs(s2), 6.501587301587302, rel_tol=1e-14)


def test_pml_beta0_reflection_choice():
    b = pml_beta0(3000.0, 40, 10.0)
    assert math.isclose(b, 3 * 3000.0 / (2 * 400.0) * math.log(1e3), rel_tol=1e-15)


def test_candidate_cost():
    c = Candidate("faber", 50, 0.01, err=1e-5, step_ms=20.0, nsteps=200)
    assert c.cost_s == pytest.approx(4.0)


class _FakeModel:
    """Records the option calls that tts.base_method makes on a model."""

    def __init__(self):
        self.window, self.form, self.lf = None, None, None

    def set_krylov_window(self, q):
        self.window = q

    def set_hork_form(self, form):
        self.form = form

    def set_leapfrog_variant(self, v):
        self.lf = v


@pytest.mark.parametrize("name,base,window,form,lf", [
    ("krylov-w2", "krylov", 2, "low-storage", None),
    ("krylov", "krylov", 0, "low-storage", None),
    ("hork-horner", "hork", 0, "horner", None),
    ("hork", "hork", 0, "low-storage", None),
    ("leapfrog-difference", "leapfrog", 0, "low-storage", 2),
    ("leapfrog", "leapfrog", 0, "low-storage", 0),
    ("faber", "faber", 0, "low-storage", None),
])
def test_candidate_names_map_to_library_methods_and_options(name, base, window, form, lf):
    from paper_2401_16322_gb300.tts import base_method
    mds = [_FakeModel(), _FakeModel()]
    assert base_method(mds, name) == base
    for md in mds:
        assert (md.window, md.form, md.lf) == (window, form, lf)


def test_single_signal_bisection_finds_the_largest_passing_step():
    """The single-signal experiment's Delta-t_max search (bisection over candidates ordered
    from the largest step down) agrees with a linear scan whenever the error grows with the
    step, and evaluates far fewer candidates."""
    from paper_2401_16322_gb300.single_signal import dt_max_search
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(1, 25))
        errs = np.sort(rng.uniform(0, 1, n))[::-1]            # largest step (first) worst
        thr = float(rng.uniform(0, 1))
        calls = []

        def ev(i):
            calls.append(i)
            return errs[i]
        got = dt_max_search(ev, list(range(n)), thr)
        passing = [i for i in range(n) if errs[i] <= thr]
        assert got == (passing[0] if passing else None)
        assert len(set(calls)) <= 2 + int(np.ceil(np.log2(n + 1)))
