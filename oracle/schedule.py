"""Oracle of automatic scheduling (Sec. 2): gates in parallel layers, idle qubits get passive noise for the
time they wait for the slowest gate of their layer.

Rule: a gate (duration >= 0) goes to the first layer after the last layer used by any of its qubits; noise
ops (duration < 0) stay right after the gate they follow.  A layer lasts max(duration of its gates).  Output per
layer: each gate with its noise, then ``idle`` on every qubit j for (layer length - time j is busy), skipped
when that is 0.
"""
from __future__ import annotations

from workloads.circuits import NativeOp


def schedule(n, ops, durations, t1, t2, idle="idle"):
    groups = []                       # [layer, [ops]]
    last = [0] * n
    for o, d in zip(ops, durations):
        if d < 0:
            groups[-1][2].append(o)
            continue
        layer = max(last[q] for q in o.qubits)
        for q in o.qubits:
            last[q] = layer + 1
        groups.append([layer, d, [o]])
    out = []
    nlayers = max((g[0] for g in groups), default=-1) + 1
    for layer in range(nlayers):
        members = [g for g in groups if g[0] == layer]
        length = max(g[1] for g in members)
        busy = [0.0] * n
        for _, d, glist in members:
            for q in glist[0].qubits:
                busy[q] = d
            out.extend(glist)
        for q in range(n):
            if length - busy[q] > 0:
                out.append(NativeOp(idle, (q,), (length - busy[q], t1[q], t2[q])))
    return out
