"""Readers of the full-size oracle results under tests/golden/ (written by make_fullsize.py)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_full(name):
    """A single-set golden file: scalar fields, Nk, bitmap digests and (optionally) the histogram."""
    g = {"digests": [], "hist": {}}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (x.strip() for x in line.split(":", 1))
            if key == "digest":
                lo, h = val.split()
                g["digests"].append((int(lo), h))
            elif key == "hist":
                v = [int(x) for x in val.split()]
                for k, c in enumerate(v[1:]):
                    g["hist"][v[0] + k] = c
            elif key == "Nk":
                g["Nk"] = [int(x) for x in val.split()]
            elif key == "S":
                g["S"] = float(val)
            else:
                g[key] = int(val)
    return g


def read_table(name):
    """A per-set golden table: one row per set, columns named in its '# columns:' line."""
    rows, cols = [], None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("# columns:"):
                cols = line.split(":", 1)[1].split()
                continue
            if line.startswith("#") or not line.strip():
                continue
            rows.append(dict(zip(cols, line.split())))
    return rows
