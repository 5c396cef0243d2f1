"""Reader for the text fixtures under tests/golden/ (values printed in the paper)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    """Return {block_name: list of text rows} from a fixture file."""
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("[") and line.endswith("]"):
                cur = line[1:-1]
                blocks[cur] = []
                continue
            blocks[cur].append(line)
    return blocks


def matrices(name):
    """Fixture blocks parsed as float matrices."""
    return {k: np.array([[float(x) for x in r.split()] for r in rows])
            for k, rows in load(name).items()}
