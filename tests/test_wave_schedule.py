"""Host check of the temporally blocked kernels' ring schedule (no GPU).

The blocked kernels keep the rows a block is working on in shared-memory
rings: the input rows copied in by TMA, the rows of every time level, the
node words and displacements, and (lambda != mu) the densities.  A launch
plan may cut a strip into segments of any number of rows, and the
calibration at create picks different cuts from run to run, so the schedule
must hold for every segment length.  This test replays the schedule the
kernels follow -- which row each level reads and writes at each sweep step,
when each input row is copied in and waited for -- with the ring sizes read
from the kernel source, and checks for every segment length that

* every row a level reads is in its ring (written earlier, not yet overwritten),
* every input row level 1 reads has been waited for,
* no ring slot is read and written in the same sweep step,
* every density the lambda != mu collision needs has been formed.
"""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2208_04088_gb300", "csrc")


def _constants():
    """Integer constants of the kernel sources (constexpr int declarations,
    single or comma-separated), evaluated in order."""
    text = open(os.path.join(CSRC, "lbm_internal.h")).read() + open(os.path.join(CSRC, "lbm_wave.cu")).read()
    text = re.sub(r"//[^\n]*", "", text)
    env = {}
    for decls in re.findall(r"constexpr int ([^;]+);", text):
        for decl in decls.split(","):
            name, _, expr = decl.partition("=")
            name, expr = name.strip(), expr.strip()
            if not re.fullmatch(r"k\w+", name) or not expr:
                continue
            try:
                env[name] = int(eval(expr.replace("/", "//"), {"__builtins__": {}}, dict(env)))
            except Exception:
                pass
    return env


C = _constants()


def _wave_schedule(Hs):
    """lambda = mu: level l computes row y = y_in0 + 1 + n - 2 (l - 1) at step n."""
    K, NI, D, NU = C["kWaveK"], C["kNI"], C["kD"], C["kNU"]
    Y0 = 1000
    y_in0 = Y0 - K
    j_last = Hs - 1 + 2 * K
    nsweep = Hs + 3 * K - 3
    errs = []
    waited = set(range(0, min(2, j_last) + 1))
    inring = {r % NI: r for r in range(0, min(D + 1, j_last) + 1)}
    nwring = {r % NU: r for r in range(0, min(D + 1, j_last) + 1)}
    lev = {}
    for n in range(nsweep):
        if n + D + 2 <= j_last:
            r = n + D + 2
            inring[r % NI] = r
            nwring[r % NU] = r
        written, read = {}, {}
        for lv in range(1, K + 1):
            lo, hi = Y0 - (K - lv), Y0 + Hs - 1 + (K - lv)
            j = 1 + n - 2 * (lv - 1)
            if not lo <= y_in0 + j <= hi:
                continue
            for r in (j - 1, j, j + 1):
                if lv == 1:
                    if r not in waited or inring.get(r % NI) != r:
                        errs.append(("input row", Hs, n, r))
                elif lev.get((lv - 1, r % 4)) != r:
                    errs.append(("level row", Hs, n, lv, r))
            if nwring.get(j % NU) != j:
                errs.append(("node-word row", Hs, n, lv, j))
            read[lv] = {r % 4 for r in (j - 1, j, j + 1)}
            if lv < K:
                written[lv] = j % 4
        for lv, slot in written.items():
            if slot in read.get(lv + 1, set()):
                errs.append(("slot read and written", Hs, n, lv))
        for lv in range(1, K):
            lo, hi = Y0 - (K - lv), Y0 + Hs - 1 + (K - lv)
            j = 1 + n - 2 * (lv - 1)
            if lo <= y_in0 + j <= hi:
                lev[(lv, j % 4)] = j
        if n + 3 <= j_last:
            waited.add(n + 3)
    return errs


def _grad_schedule(Hs):
    """lambda != mu: level l collides row y = y_in0 - 1 + n - skew (l - 1) and
    forms the densities of row y + 2 at step n."""
    K, S = C["kWaveGradK"], C["kGradSkew"]
    NI, D, NL, ND, NU = C["kGradNI"], C["kGradD"], C["kGradNL"], C["kGradND"], C["kGradNU"]
    Y0 = 1000
    y_in0 = Y0 - 2 * K
    j_last = Hs + 4 * K - 1
    nsweep = Hs + 6 * K - 3
    errs = []
    waited = set(range(0, min(2, j_last) + 1))
    inring = {r % NI: r for r in range(0, min(D + 1, j_last) + 1)}
    nwring = {r % NU: r for r in range(0, min(D + 1, j_last) + 1)}
    lev, den = {}, {}
    for n in range(nsweep):
        if n + D + 2 <= j_last:
            r = n + D + 2
            inring[r % NI] = r
            nwring[r % NU] = r
        written, read = {}, {}
        for lv in range(1, K + 1):
            lo, hi = Y0 - 2 * (K - lv), Y0 + Hs - 1 + 2 * (K - lv)
            j = -1 + n - S * (lv - 1)
            need, words = [], []
            if lo - 1 <= y_in0 + j + 2 <= hi + 1:
                need += [j + 1, j + 2, j + 3]
                words.append(j + 2)
            if lo <= y_in0 + j <= hi:
                need += [j - 1, j, j + 1]
                words.append(j)
                for r in (j - 1, j + 1):
                    if den.get((lv, r % ND)) != r:
                        errs.append(("density row", Hs, n, lv, r))
            for r in need:
                if lv == 1:
                    if r not in waited or inring.get(r % NI) != r:
                        errs.append(("input row", Hs, n, r))
                elif lev.get((lv - 1, r % NL)) != r:
                    errs.append(("level row", Hs, n, lv, r))
            for r in words:
                if nwring.get(r % NU) != r:
                    errs.append(("node-word row", Hs, n, lv, r))
            read[lv] = {r % NL for r in need}
            if lo <= y_in0 + j <= hi and lv < K:
                written[lv] = j % NL
        for lv, slot in written.items():
            if slot in read.get(lv + 1, set()):
                errs.append(("slot read and written", Hs, n, lv))
        for lv in range(1, K + 1):
            lo, hi = Y0 - 2 * (K - lv), Y0 + Hs - 1 + 2 * (K - lv)
            j = -1 + n - S * (lv - 1)
            if lo - 1 <= y_in0 + j + 2 <= hi + 1:
                den[(lv, (j + 2) % ND)] = j + 2
            if lo <= y_in0 + j <= hi and lv < K:
                lev[(lv, j % NL)] = j
        if n + 3 <= j_last:
            waited.add(n + 3)
    return errs


def test_constants_found():
    for k in ("kWaveK", "kNI", "kD", "kNU", "kWaveGradK", "kGradSkew", "kGradNI", "kGradD",
              "kGradNL", "kGradND", "kGradNU"):
        assert k in C, k


@pytest.mark.parametrize("Hs", range(1, 70))
def test_wave_schedule_holds_for_every_segment_length(Hs):
    assert _wave_schedule(Hs) == []


@pytest.mark.parametrize("Hs", range(1, 70))
def test_grad_schedule_holds_for_every_segment_length(Hs):
    assert _grad_schedule(Hs) == []


def test_schedule_check_catches_a_short_ring():
    # the check is not vacuous: a node-word ring two rows short breaks the lambda = mu schedule
    saved = dict(C)
    try:
        C["kNU"] = C["kNU"] - 2
        assert any(_wave_schedule(Hs) for Hs in (1, 5, 20))
    finally:
        C.clear()
        C.update(saved)
