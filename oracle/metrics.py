"""Error measures of Sec. 5.1 (L2-err and max-err of the computed solution against the exact one).

The rel-res of Sec. 5.1, ||F - A U||_2 / ||F - A U^0||_2, is evaluated where it is used (oracle.gmres and
the tests), not here.
"""
import numpy as np


def l2_err(u, U):
    return np.linalg.norm((u - U).ravel()) / np.linalg.norm(u.ravel())


def max_err(u, U):
    return np.abs(u - U).max()
