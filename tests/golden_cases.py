"""Loader for the hand-worked examples in ``tests/golden/hand_examples.txt``."""

import os
from typing import List, NamedTuple, Tuple

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


class Case(NamedTuple):
    name: str
    text: bytes
    patterns: List[bytes]
    expect: List[Tuple[int, int]]


def load_hand_examples() -> List[Case]:
    cases: List[Case] = []
    cur = None
    with open(os.path.join(GOLDEN, "hand_examples.txt")) as f:
        for raw in f:
            line = raw.rstrip("\n")
            if not line.strip() or line.lstrip().startswith("#"):
                continue
            key, _, val = line.partition(":")
            val = val[1:] if val.startswith(" ") else val
            if key == "case":
                cur = Case(val.strip(), b"", [], [])
                cases.append(cur)
            elif key == "text":
                cases[-1] = cur = cur._replace(text=val.encode())
            elif key == "text_hex":
                cases[-1] = cur = cur._replace(text=bytes.fromhex(val.strip()))
            elif key == "pattern":
                cur.patterns.append(val.encode())
            elif key == "pattern_hex":
                cur.patterns.append(bytes.fromhex(val.strip()))
            elif key == "expect":
                a, b = val.split()
                cur.expect.append((int(a), int(b)))
            else:
                raise ValueError(f"bad golden line: {line!r}")
    return cases
