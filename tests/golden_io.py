"""Readers for the text fixtures under tests/golden (values printed in the paper)."""

import math
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_PHI = (1 + math.sqrt(5)) / 2
_NAMES = {"sqrt": math.sqrt, "phi": _PHI, "__builtins__": {}}


def value(tok: str) -> float:
    if tok == ".":
        return 0.0
    return float(eval(tok, dict(_NAMES)))  # tokens are short arithmetic literals from the paper


def lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for ln in fh:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln


def matrix(name):
    return [[value(t) for t in ln.split()] for ln in lines(name)]
