"""Reader for the small text fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_COMPOUND = ("iter", "edges", "fixed")


def read(name):
    """Returns {key: [tokens]} for lines 'key tok tok ...' ('#' starts a
    comment).  A line 'graph edges ...' or 'graph iterN ...' has the two-word
    key 'graph edges' / 'graph iterN'."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            parts = line.split("#", 1)[0].split()
            if not parts:
                continue
            if len(parts) > 1 and parts[1].startswith(_COMPOUND):
                out[parts[0] + " " + parts[1]] = parts[2:]
            else:
                out[parts[0]] = parts[1:]
    return out


def edges(tokens):
    s, d = [], []
    for t in tokens:
        a, b = t.split("-")
        s.append(int(a))
        d.append(int(b))
    return s, d
