"""Plain reader of text detector error models (test infrastructure).

The checker for the library's DEM reader: it turns the same text into the
decoding problem (H, A, p) of App. A with a different method (line by line,
recursion on repeat blocks, dense 0/1 matrices) and shares nothing with it.
Semantics: one column per error(p) line in the order met (repeat blocks
expanded); detector indices offset by the running shift_detectors total; a
mechanism flips the XOR of its D/L targets ('^' only separates parts);
M / K are one more than the largest detector / observable index met or
declared; with merge, mechanisms with equal (detector, observable) sets
become one with probability p1 (1 - p2) + p2 (1 - p1).
"""
from __future__ import annotations

import re

import numpy as np

_STMT = re.compile(r"^([A-Za-z_][A-Za-z0-9_]*)(\[[^\]]*\])?(\(([^)]*)\))?(.*)$")


def _lines(text: str):
    out = []
    for raw in text.splitlines():
        s = raw.split("#", 1)[0].strip()
        if s:
            out.append(s)
    return out


def _parse(lines, i):
    """Statements from lines[i:] until a closing brace; returns (stmts, next index)."""
    stmts = []
    while i < len(lines):
        s = lines[i]
        if s == "}":
            return stmts, i + 1
        m = _STMT.match(s)
        if not m:
            raise ValueError(f"bad line: {s}")
        name, args, rest = m.group(1), m.group(4), m.group(5).strip()
        body = None
        if rest.endswith("{"):
            rest = rest[:-1].strip()
            body, i = _parse(lines, i + 1)
        else:
            i += 1
        stmts.append((name, [float(a) for a in args.split(",")] if args else [], rest.split(), body))
    return stmts, i


def read_dem(text: str, merge: bool = False) -> dict:
    stmts, _ = _parse(_lines(text), 0)
    cols, probs = [], []
    state = {"shift": 0, "max_d": -1, "max_l": -1}

    def run(block):
        for name, args, targets, body in block:
            if name == "error":
                dets, obs = set(), set()
                for t in targets:
                    if t == "^":
                        continue
                    k = int(t[1:])
                    if t[0] == "D":
                        dets ^= {state["shift"] + k}
                    else:
                        obs ^= {k}
                cols.append((frozenset(dets), frozenset(obs)))
                probs.append(args[0])
                state["max_d"] = max([state["max_d"], *dets])
                state["max_l"] = max([state["max_l"], *obs])
            elif name == "detector":
                for t in targets:
                    state["max_d"] = max(state["max_d"], state["shift"] + int(t[1:]))
            elif name == "logical_observable":
                for t in targets:
                    state["max_l"] = max(state["max_l"], int(t[1:]))
            elif name == "shift_detectors":
                state["shift"] += int(targets[0])
            elif name == "repeat":
                for _ in range(int(targets[0])):
                    run(body)
            else:
                raise ValueError(f"unknown instruction {name}")

    run(stmts)
    if merge:
        seen, mc, mp = {}, [], []
        for c, p in zip(cols, probs):
            if c in seen:
                q = mp[seen[c]]
                mp[seen[c]] = q * (1 - p) + p * (1 - q)
            else:
                seen[c] = len(mc)
                mc.append(c)
                mp.append(p)
        cols, probs = mc, mp
    M, K, N = state["max_d"] + 1, state["max_l"] + 1, len(cols)
    H = np.zeros((M, N), np.uint8)
    A = np.zeros((K, N), np.uint8)
    for j, (d, o) in enumerate(cols):
        for i in d:
            H[i, j] = 1
        for i in o:
            A[i, j] = 1
    return {"M": M, "N": N, "K": K, "H": H, "A": A, "priors": np.array(probs, np.float64)}
