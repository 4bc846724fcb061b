"""Writes the inputs of the Eq. 1 enforcement pins (tests/test_oracle_enforcement.py):

  escalation_1d.txt  one-brick 1D fields whose second component is coded
                     CODED only after lowering its lowest plane (escalation,
                     rule R13);
  r14_ties_1d.txt    one-brick 1D fields whose first component codes CODED in
                     exactly as many bits as RAW storage (rule R14: a tie
                     keeps CODED).

Run from the repository root: python tests/golden/find_enforcement_cases.py
It calls only the CPU oracle (oracle/), on seeded random bricks.  The stored
values are inputs, not expected results: the tests recompute what the coder
must do from its separately pinned unit steps.

Escalation search: four values of mixed magnitude, a coarse first tolerance,
and a second tolerance set to an exact power of two 2^(p + c - s) for the
block exponent of the residual the first component leaves (s = P - 2 - 2d -
emax, c = 1 for d = 1), where the floating-point sum of Eq. 1 is most likely
to land one unit off.  Tie search: random bricks at random tolerances.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

MODE_CODED = 1


def _bits_of(x, dt):
    return ",".join("%x" % int(b) for b in x.view(np.uint32 if dt == np.float32 else np.uint64))


def escalations(dt, seed, want, limit=400000):
    P = 32 if dt == np.float32 else 64
    Q, c = P - 4, 1
    emin = -125 if dt == np.float32 else -1021
    rng = np.random.default_rng(seed)
    hits = []
    for _ in range(limit):
        x = (rng.normal(size=4) * 2.0 ** rng.uniform(-3, 3, size=4)).astype(dt)
        t1 = float(2.0 ** rng.uniform(-5, 0) * np.max(np.abs(x)))
        _, _, xt1, _ = O.code_brick(x, [t1], 0)
        e = x.astype(np.float64) - xt1
        nz = np.abs(e[e != 0])
        if len(nz) == 0:
            continue
        emax = max(int(np.frexp(nz.max())[1]), emin)
        p = int(rng.integers(1, 9))
        t2 = 2.0 ** (p + c - (Q - emax))
        if not t2 < t1:
            continue
        _, _, _, st = O.code_brick(x, [t1, t2], 0)
        if st[1, O.ST_ESC] > 0:
            hits.append((x, t1, t2))
            if len(hits) == want:
                break
    return hits


def ties(dt, seed, want, limit=400000):
    P = 32 if dt == np.float32 else 64
    len_raw = 2 + 4 * P
    rng = np.random.default_rng(seed)
    hits = []
    for _ in range(limit):
        x = (rng.normal(size=4) * 2.0 ** rng.uniform(-2, 2, size=4)).astype(dt)
        t = float(2.0 ** -rng.uniform(10, 60 if dt == np.float64 else 28))
        bits, nbits, _, _ = O.code_brick(x, [t], 0)
        if nbits[0] == len_raw and (int(bits[0, 0]) & 3) == MODE_CODED:
            hits.append((x, t))
            if len(hits) == want:
                break
    return hits


def main():
    lines = ["# One-brick 1D fields (4 values) whose component 2 is coded CODED after escalation.",
             "# Written by tests/golden/find_enforcement_cases.py, which calls only the CPU oracle.",
             "# columns: dtype | x[0..3] as IEEE bit patterns (hex) | tau_1 tau_2 (hex doubles)"]
    for dt, name, seed in ((np.float32, "f32", 11), (np.float64, "f64", 12)):
        for x, t1, t2 in escalations(dt, seed, 3):
            lines.append("%s | %s | %s %s" % (name, _bits_of(x, dt), t1.hex(), t2.hex()))
    with open(os.path.join(HERE, "escalation_1d.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    lines = ["# One-brick 1D fields (4 values) whose one component codes CODED in exactly 2 + 4P bits,",
             "# the length of RAW storage.",
             "# Written by tests/golden/find_enforcement_cases.py, which calls only the CPU oracle.",
             "# columns: dtype | x[0..3] as IEEE bit patterns (hex) | tau_1 (hex double)"]
    for dt, name, seed in ((np.float32, "f32", 21), (np.float64, "f64", 22)):
        for x, t in ties(dt, seed, 2):
            lines.append("%s | %s | %s" % (name, _bits_of(x, dt), t.hex()))
    with open(os.path.join(HERE, "r14_ties_1d.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
