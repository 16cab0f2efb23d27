"""Reader for paper_values.txt (values printed in the paper, with their citation)."""
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def paper_values():
    out = {}
    with open(os.path.join(_HERE, "paper_values.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, cite = line.split(None, 2)
            out[name] = (float(value), cite)
    return out
