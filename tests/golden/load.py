"""Reader for the hand-worked fixtures in this folder (plain text: '#'
comments, 'key value' scalars, and matrices introduced by a key line)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name: str) -> dict:
    out = {}
    key = None
    rows = []
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if len(parts) == 1 and not parts[0].lstrip("-").isdigit():
                if key is not None and rows:
                    out[key] = np.array(rows, dtype=np.int64)
                key, rows = parts[0], []
            elif len(parts) == 2 and not parts[0].lstrip("-").isdigit():
                if key is not None and rows:
                    out[key] = np.array(rows, dtype=np.int64)
                    key, rows = None, []
                out[parts[0]] = int(parts[1])
            else:
                rows.append([int(x) for x in parts])
    if key is not None and rows:
        out[key] = np.array(rows, dtype=np.int64)
    return out
