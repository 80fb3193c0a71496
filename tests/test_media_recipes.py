"""The seeded scattering workloads follow their stated recipe (CPU): the incident field is a plane wave of
wavenumber k0 along a unit direction (read back from f = -(k^2 - k0^2) u_inc), k0 = 2 pi n / ppw, the media
of the bench and the batches are real (no attenuation), the layered medium stays within its contrast range,
the sphere of Sec. 5.2 takes its two printed values, and every generator is deterministic in its seeds."""
import math

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2602_07711_gb300 import media

N = 24


def _incident(k2, f, k0):
    """u_inc = f / (-(k^2 - k0^2)) wherever the medium differs from the background (a quotient of the
    product that formed f, so exact to rounding however small the difference)."""
    dk = k2 - k0 * k0
    m = dk != 0
    u = np.full(f.shape, np.nan + 0j)
    u[m] = f[m] / -dk[m]
    return u, m


def _direction_from_phase(u, k0, h):
    """Phase increments of a plane wave along x, y, z (axes 2, 1, 0 of [z, y, x]) over one grid step."""
    out = []
    for ax in (2, 1, 0):
        hi, lo = np.take(u, range(1, u.shape[ax]), axis=ax), np.take(u, range(0, u.shape[ax] - 1), axis=ax)
        ok = np.isfinite(hi) & np.isfinite(lo)
        r = hi[ok] / lo[ok]
        ang = np.angle(r)
        assert np.ptp(ang) < 1e-9                      # the same increment everywhere: a plane wave
        out.append(ang.mean() / (k0 * h))
    return np.array(out)


@pytest.mark.parametrize("seeds", [(3, 4), (1, 2), (11, 12)])
def test_bumps_incident_wave_is_a_unit_direction_plane_wave(seeds):
    k2, f, k0 = media.bumps(N, *seeds, ppw=10.0, contrast=0.3)
    assert k2.shape == (N, N, N) and k2.dtype == np.complex128 and f.dtype == np.complex128
    assert math.isclose(k0, 2 * math.pi * N / 10.0, rel_tol=1e-15)
    assert np.all(k2.imag == 0)                        # no attenuation: the real-medium kernels apply
    u, m = _incident(k2, f, k0)
    assert m.mean() > 0.3
    assert np.allclose(np.abs(u[m]), 1.0, atol=1e-12)
    d = _direction_from_phase(u, k0, 1.0 / N)
    assert abs(np.linalg.norm(d) - 1.0) < 1e-9
    assert np.allclose(d, media.direction(seeds[1]), atol=1e-9)


def test_generators_are_deterministic_in_their_seeds():
    a = media.bumps(N, 3, 4)
    b = media.bumps(N, 3, 4)
    c = media.bumps(N, 5, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    la, lb = media.layered(N, 5), media.layered(N, 5)
    assert np.array_equal(la[0], lb[0]) and np.array_equal(la[1], lb[1])


def test_layered_medium_stays_within_its_contrast_range():
    k2, f, k0 = media.layered(32, 5, ppw=8.0, lo=0.7, hi=1.3)
    rel = k2.real / (k0 * k0)
    assert np.all(k2.imag == 0) and rel.min() >= 0.7 - 1e-12 and rel.max() <= 1.3 + 1e-12
    assert math.isclose(k0, 2 * math.pi * 32 / 8.0, rel_tol=1e-15)
    # eight horizontal layers: away from the spheres, each z-plane is constant
    planes = [np.unique(rel[z]) for z in range(32)]
    assert min(len(p) for p in planes) == 1


def test_sphere_takes_the_printed_values():
    n = 40
    k2, f, k0 = media.sphere(n)
    vals = set(np.unique(k2).tolist())
    assert vals == {complex(1050, 2.26), complex(439.2, 0)}
    assert math.isclose(k0 * k0, 439.2, rel_tol=1e-14)
    frac = np.mean(k2 == complex(1050, 2.26))
    assert abs(frac - 4.0 / 3.0 * math.pi * 0.1 ** 3) < 0.25 * 4.0 / 3.0 * math.pi * 0.1 ** 3
    u, m = _incident(k2, f, k0)                        # f vanishes outside; inside it is a +z plane wave
    assert np.all(f[~m] == 0) and np.allclose(np.abs(u[m]), 1.0, atol=1e-12)
