"""Reader of ``paper_claims.txt`` (values printed in the paper, each cited there)."""
import os


def load():
    out = {}
    path = os.path.join(os.path.dirname(__file__), "paper_claims.txt")
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split("=", 1))
            out[key] = val
    return out
