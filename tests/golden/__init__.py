"""Fixtures of values printed in the paper (each file cites its source)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def table2_asyrk():
    """Rows (m, n, delta, seconds, epochs) of Section 5, Table 2 (AsyRK columns)."""
    rows = []
    with open(os.path.join(HERE, "table2_asyrk.txt")) as f:
        for ln in f:
            ln = ln.split("#", 1)[0].split()
            if ln:
                rows.append((int(ln[0]), int(ln[1]), float(ln[2]), float(ln[3]), int(ln[4])))
    return rows
