"""Readers of the paper's printed tables (text fixtures under tests/golden/, each citing its table)."""
import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def high_order_rows():
    """Tables tab:fourth_order_results / tab:sixth_order_results: (order, N, max-err as printed, L2-err, N0)."""
    rows = []
    with open(os.path.join(GOLDEN, "high_order_table.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                order, n, me, l2, n0 = line.split()
                rows.append((int(order), int(n), me, float(l2), int(n0)))
    return rows


def printed_half_unit(text):
    """Half a unit in the last printed digit of a table entry ('0.02' -> 0.005, '7.64e-03' -> 5e-6)."""
    mant, _, exp = text.lower().partition("e")
    decimals = len(mant.split(".")[1]) if "." in mant else 0
    return 0.5 * 10.0 ** (-decimals + (int(exp) if exp else 0))
