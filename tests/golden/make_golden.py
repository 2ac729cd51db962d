"""Writes the stored expected values under tests/golden/ (calls only oracle/).

fd_weights_no6.txt: Eq. (weightsLap), Sec. 3.1, for n_o = 6, as exact rationals of
h^2 w_p, p = 0..6.
fd_grad_weights_no6.txt: the weights of Eq. (gradient:approximate), Sec. 3.1, for
n_o = 6, as exact rationals of h w~_p, p = 1..6.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lap_weights_exact  # noqa: E402
from oracle.observables import grad_weights_exact  # noqa: E402


def main():
    w = lap_weights_exact(6)
    with open(os.path.join(HERE, "fd_weights_no6.txt"), "w") as f:
        f.write("# h^2 * w_p for p = 0..6, Eq. (weightsLap), Sec. 3.1 (n_o = 6), exact rationals\n")
        for p, x in enumerate(w):
            f.write(f"{p} {x.numerator} {x.denominator}\n")
    with open(os.path.join(HERE, "fd_grad_weights_no6.txt"), "w") as f:
        f.write("# h * w~_p for p = 1..6, Eq. (gradient:approximate), Sec. 3.1 (n_o = 6), "
                "exact rationals\n")
        for p, x in enumerate(grad_weights_exact(6), start=1):
            f.write(f"{p} {x.numerator} {x.denominator}\n")


if __name__ == "__main__":
    main()
