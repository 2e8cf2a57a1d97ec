"""The double-precision parity rule shared by the GPU parity tests.

The CUDA decoder computes in single precision and matches the oracle's
single-precision build bit for bit (checked on every shot elsewhere).
Against the double-precision oracle a shot may differ only where the two
precisions take a different decision for a reason rounding explains: the
first decision on which the double- and single-precision runs of the shot
differ (their decision logs, compared record by record) must be preceded,
or taken, by a decision of the double-precision run whose relative margin is
below the guard band of 1e-4 (the LLR bar) or that is an exact tie.  Counts
are reported at that guard band and at the 1e-6 near-tie threshold.
"""
import numpy as np

import oracle
from paper_2512_07057_gb300 import workloads as W

GUARD = 1e-4
NEAR_TIE = 1e-6


def explain_mismatches(prob, op, syndromes, idx):
    """For each shot index in idx: (first divergent record, near tie at
    1e-6 before it, at 1e-4 before it, the record's (call, kind, iteration))."""
    if len(idx) == 0:
        return []
    g64, g32 = oracle.Graph(prob, "f64"), oracle.Graph(prob, "f32")
    s_all = W.unpack_bits(np.asarray(syndromes)[idx], prob.M)
    out = []
    for s in s_all:
        l64 = g64.decode_log(s, op)["log"]
        l32 = g32.decode_log(s, op)["log"]
        k = oracle.first_divergence(l64, l32)
        at = (int(l64["call"][k]), int(l64["kind"][k]), int(l64["t"][k])) if 0 <= k < len(l64["key"]) else None
        out.append((k, oracle.near_tie_before(l64, k, NEAR_TIE) if k >= 0 else False,
                    oracle.near_tie_before(l64, k, GUARD) if k >= 0 else False, at))
    return out


def check_against_f64(prob, op, syndromes, gpu, nthreads=8, ref64=None, max_extra=2, max_frac=1e-3):
    """Compare GPU outputs (corrections, status) with the double-precision
    oracle on the same shots under the rule above; returns the counts."""
    if ref64 is None:
        ref64 = oracle.Graph(prob, "f64").decode_batch(syndromes, op, nthreads=nthreads)
    diff = (gpu["corrections"] != ref64["corrections"]).any(1) | (gpu["status"] != ref64["status"])
    bad = np.nonzero(diff)[0]
    info = explain_mismatches(prob, op, syndromes, bad)
    unexplained = [int(b) for b, (k, _, g4, _) in zip(bad, info) if k < 0 or not g4]
    counts = dict(shots=int(len(diff)), mismatches=int(len(bad)),
                  near_tie_1e6=int(sum(1 for x in info if x[1])),
                  near_tie_1e4=int(sum(1 for x in info if x[2])))
    print(f"f64 parity: {counts}; divergences (call, kind, t): {[x[3] for x in info][:10]}")
    assert not unexplained, f"f64 mismatches with no near tie before the divergence: shots {unexplained[:10]}"
    assert len(bad) <= max_extra + max_frac * len(diff), f"{len(bad)} f64 mismatches"
    return counts, ref64
