"""Error and residual measures of Sec. 5.1."""
import numpy as np


def rel_res(AU, F, AU0):
    return np.linalg.norm((AU - F).ravel()) / np.linalg.norm((AU0 - F).ravel())


def relmax_res(AU, F, AU0):
    return np.abs(AU - F).max() / np.abs(AU0 - F).max()


def l2_err(u, U):
    return np.linalg.norm((u - U).ravel()) / np.linalg.norm(u.ravel())


def max_err(u, U):
    return np.abs(u - U).max()


def relmax_err(u, U):
    return np.abs(u - U).max() / np.abs(u).max()
