"""Readers of the paper's printed values in tests/golden/ (each file cites
the table or section it comes from)."""
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def table1():
    """{T: {"r_e", "r_mx", "r_my", "r_mz", "r_amz"}} with None for empty entries."""
    keys = ("r_e", "r_mx", "r_my", "r_mz", "r_amz")
    return {float(r[0]): {k: (None if v == "---" else float(v)) for k, v in zip(keys, r[1:])}
            for r in _rows("table1_distribution_coefficients.txt")}


def critical_temperature(model):
    """(L_small, L_large, T_C, error) for 'heisenberg_sc' or 'ising_square'."""
    for r in _rows("critical_temperatures.txt"):
        if r[0] == model:
            return int(r[1]), int(r[2]), float(r[3]), float(r[4])
    raise KeyError(model)
