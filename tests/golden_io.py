"""Parser for the hand-derived golden cases in tests/golden/*.case."""
import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_case(path):
    names, stream, ep, expect = {}, [], None, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, val = line.partition(":")
        val = val.strip()
        if key == "types":
            for tok in val.split():
                nm, _, idx = tok.partition("=")
                names[nm] = int(idx)
        elif key == "stream":
            for tok in val.split():
                nm, _, t = tok.partition("@")
                stream.append((names[nm], int(t)))
        elif key == "episode":
            parts = [p.strip() for p in val.split("|")]
            E = [names[x] for x in parts[0].split()]
            lo = [int(x) for x in parts[1].split()[1:]]
            hi = [int(x) for x in parts[2].split()[1:]]
            ep = (E, lo, hi)
        elif key == "expect":
            expect = int(val)
    types = np.array([s[0] for s in stream], np.uint16)
    times = np.array([s[1] for s in stream], np.int32)
    return os.path.basename(path), types, times, ep, expect


def all_cases():
    return [load_case(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.case")))]
