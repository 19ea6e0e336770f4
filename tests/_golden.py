"""Loader for the hand-worked cases in tests/golden/hand_cases.txt."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_hand_cases(path=os.path.join(GOLDEN, "hand_cases.txt")):
    cases, cur, block = [], None, None
    with open(path) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            head, *rest = line.split()
            if head == "case":
                cur = {"name": rest[0], "mask": [], "marker": [], "expected": []}
                block = None
            elif head == "conn":
                cur["conn"] = [int(c) for c in rest]
            elif head == "op":
                cur["op"] = rest[0]
            elif head == "dtype":
                cur["dtype"] = {"u8": np.uint8, "u16": np.uint16}[rest[0]]
            elif head in ("mask", "marker", "expected"):
                block = head
            elif head == "end":
                for k in ("mask", "marker", "expected"):
                    cur[k] = np.array(cur[k], dtype=cur["dtype"])
                cases.append(cur)
                cur = block = None
            else:
                cur[block].append([int(v) for v in line.split()])
    return cases
