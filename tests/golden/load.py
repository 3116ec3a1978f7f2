"""Reader of the paper-value fixtures in this folder (plain text, one key per line)."""
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def paper_values(name="paper_examples.txt"):
    out = {}
    with open(os.path.join(_HERE, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kv = line.split("|")[0]
            k, v = kv.split("=", 1)
            out[k.strip()] = v.strip()
    return out
