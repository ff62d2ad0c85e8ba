"""Reader for the hand-worked fixtures under tests/golden/."""
import glob
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    path = os.path.join(GOLDEN, name)
    d = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            d[key] = rest.split()
    n = int(d["n"][0])
    pairs = [tuple(int(x) for x in e.split("-")) for e in d.get("edges", [])]
    p, q = (int(x) for x in d["eps"][0].split("/"))
    out = {
        "name": name, "n": n, "pairs": pairs, "p": p, "q": q,
        "rounds": int(d["rounds"][0]), "best_round": int(d["best_round"][0]),
        "E": int(d["E"][0]), "V": int(d["V"][0]),
        "hist_S": np.array([int(x) for x in d["hist_S"]], np.uint64),
        "hist_E": np.array([int(x) for x in d["hist_E"]], np.uint64),
        "peel_round": np.array([int(x) for x in d["peel_round"]], np.uint32),
        "core": np.array([int(x) for x in d["core"]], np.uint32),
    }
    return out


def all_fixtures(prefix="bahmani_"):
    return sorted(os.path.basename(p) for p in glob.glob(os.path.join(GOLDEN, prefix + "*.txt")))


def load_cbds(name):
    d = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            d[key] = rest.split()
    pairs = [tuple(int(x) for x in e.split("-")) for e in d.get("edges", [])]
    return {
        "name": name, "n": int(d["n"][0]), "pairs": pairs,
        "core": np.array([int(x) for x in d["core"]], np.uint32),
        "densest_core": tuple(int(x) for x in d["densest_core"]),
        "phase2": tuple(int(x) for x in d["phase2"]),
    }
