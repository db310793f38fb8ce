"""Write the FC(Gram) continuation tables used by the tests.

Calls only the oracle (oracle.fc.gram_table, 80-digit arithmetic) and stores
E (n_cont x 2*n_match, right-wall block first) as text, one row per line, so
that GPU-box tests need no multiprecision library.  Run from the repo root:

    python tests/golden/make_fc_gram.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.fc import gram_table  # noqa: E402

CASES = [(5, 22), (5, 24), (5, 25), (5, 26), (5, 28), (5, 32)]


def path(n_match, n_cont):
    return os.path.join(HERE, f"fc_gram_d{n_match}_c{n_cont}.txt")


def main():
    for d, c in CASES:
        E = gram_table(d, c)
        with open(path(d, c), "w") as f:
            f.write(f"# FC(Gram) table, n_match={d} n_cont={c}; written by make_fc_gram.py from oracle.fc.gram_table\n")
            for row in E:
                f.write(" ".join(repr(float(x)) for x in row) + "\n")


if __name__ == "__main__":
    main()
