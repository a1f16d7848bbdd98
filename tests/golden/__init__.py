"""Stored values the paper states, each with its citation (see paper_facts.txt)."""

import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def load_facts():
    out = {}
    with open(os.path.join(_HERE, "paper_facts.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = line.split()
            out[key] = float(val)
    return out
