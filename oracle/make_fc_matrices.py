"""Write the oracle's FC matrices (Q, R, A, A_r, singular values, residuals) to
tests/golden, so that tests need not redo the 50-digit computation each run.

Calls only ``oracle``.  Usage: python -m oracle.make_fc_matrices [d C Z n_os n_r m_F]
"""
import sys

from oracle.fc_matrices import compute_fc_matrices, golden_path, save_fc_matrices


def main(argv):
    vals = [int(a) for a in argv] if argv else [5, 27, 12, 20, 6, 20]
    d, C, Z, n_os, n_r, m_F = vals
    mats = compute_fc_matrices(d, C, Z, n_os, n_r, m_F)
    path = golden_path(d, C, Z, n_os, n_r, m_F)
    save_fc_matrices(mats, path)
    print(path, "sv range %.3e .. %.3e" % (mats["sv"][0], mats["sv"][-1]),
          "max resid %.2e" % mats["resid"].max())


if __name__ == "__main__":
    main(sys.argv[1:])
