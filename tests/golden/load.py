"""Reader for the small text fixtures in this folder (sections in [brackets])."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def read(name: str) -> dict:
    out, cur = {}, None
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("[") and line.endswith("]"):
                cur = line[1:-1]
                out[cur] = []
                continue
            out[cur].append([float(t) for t in line.split()])
    return {k: np.array(v) for k, v in out.items()}
