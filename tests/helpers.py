"""Shared test helpers: tolerances and comparison against the oracle."""
import numpy as np

U = 2.0 ** -53


def bound(k, absprod):
    """The acceptance bound |C - C_dot2| <= 2 k u (|A||B|)."""
    return 2.0 * max(k, 1) * U * absprod


def assert_within_bound(C, ref, absprod, k, what=""):
    C = np.asarray(C)
    err = np.abs(C - ref)
    lim = bound(k, absprod)
    bad = ~(err <= lim)
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(
            f"{what}: {int(bad.sum())} entries outside 2ku|A||B|; first at {tuple(i)}: "
            f"got {C[tuple(i)]!r} ref {ref[tuple(i)]!r} err {err[tuple(i)]:.3e} lim {lim[tuple(i)]:.3e}")
    return float(np.max(err / np.where(lim > 0, lim, 1.0))) if C.size else 0.0


def assert_bitwise(C, ref, what=""):
    C = np.asarray(C)
    ref = np.asarray(ref)
    assert C.shape == ref.shape, (C.shape, ref.shape)
    same = (C == ref) | (np.isnan(C) & np.isnan(ref))
    if not same.all():
        i = np.argwhere(~same)[0]
        raise AssertionError(f"{what}: {int((~same).sum())} entries differ; first at {tuple(i)}: "
                             f"got {C[tuple(i)]!r} ref {ref[tuple(i)]!r}")
