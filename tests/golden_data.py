"""Reader of the text fixtures under tests/golden/: sections `[name]`, a header row of column names, then
one row per item (first column its name, the others numbers); `#` starts a comment line."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(fname: str) -> dict:
    """{section: {row name: {column: value}}}"""
    out, sec, cols = {}, None, None
    with open(os.path.join(GOLDEN, fname)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("[") and line.endswith("]"):
                sec, cols = line[1:-1], None
                out[sec] = {}
                continue
            parts = line.split()
            if cols is None:
                cols = parts[1:]
                continue
            if len(parts) != len(cols) + 1:
                raise ValueError(f"{fname} [{sec}]: row {parts[0]} has {len(parts) - 1} values, {len(cols)} columns")
            out[sec][parts[0]] = {c: float(v) for c, v in zip(cols, parts[1:])}
    return out
