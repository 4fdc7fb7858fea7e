"""Reader for the small text fixtures under tests/golden/."""
import os

_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_values():
    out = {}
    with open(os.path.join(_DIR, "paper_printed_values.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split()[:2]
            out[key] = float(val)
    return out
