"""Reads tests/golden/paper_constants.txt (numbers printed in the paper)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_constants.txt")


def constants():
    out = {}
    with open(_PATH) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value = line.split()[:2]
            out[name] = float(value)
    return out
