"""Host check of the instance-major dense schedule's algebra (dense_im.cu).

The kernels factorise each instance's dense block left-looking by outer
panels of 128: the block column and row of outer panel j first take the
products of all earlier panels (k_im_gemm, depth 128 j); then two 64-wide
steps each factorise a 64 x 64 diagonal block together with the inverses of
its factors (k_im_diag) and multiply the rows below / columns to the right by
those inverses (k_im_panel), the second step first subtracting its product
with the first step's L and U.  This test replays that sequence of block
operations in float64 with numpy, region by region, and checks it against an
unblocked LU without pivoting (Sec. 4.3's dense tail), on block sizes with and
without a last outer panel of 64.  It pins the schedule, not the kernels: the
GPU parity tests compare the kernels with the oracle.
"""
import numpy as np
import pytest


def plain_lu(a):
    """Doolittle LU without pivoting, L unit lower and U in one array."""
    a = a.copy()
    n = a.shape[0]
    for p in range(n - 1):
        a[p + 1:, p] /= a[p, p]
        a[p + 1:, p + 1:] -= np.outer(a[p + 1:, p], a[p, p + 1:])
    return a


def diag_step(a, ki):
    """LU of the 64 x 64 block at (ki, ki) and the inverses of its factors."""
    d = plain_lu(a[ki:ki + 64, ki:ki + 64])
    a[ki:ki + 64, ki:ki + 64] = d
    lo = np.tril(d, -1) + np.eye(64)
    up = np.triu(d)
    return np.linalg.inv(up), np.linalg.inv(lo)


def schedule_lu(a0, drop_row_update=False):
    a = a0.copy()
    n = a.shape[0]
    assert n % 64 == 0
    for kj in range(0, n, 128):
        if kj > 0:
            # block column and row of panel kj minus the products of panels 0 .. j-1
            c = min(128, n - kj)
            a[kj:, kj:kj + c] -= a[kj:, :kj] @ a[:kj, kj:kj + c]
            if not drop_row_update:
                a[kj:kj + c, kj + 128:] -= a[kj:kj + c, :kj] @ a[:kj, kj + 128:]
        # step 0 at ki = kj
        ui, li = diag_step(a, kj)
        a[kj + 64:, kj:kj + 64] = a[kj + 64:, kj:kj + 64] @ ui        # L21 = A21 U11^-1
        a[kj:kj + 64, kj + 64:] = li @ a[kj:kj + 64, kj + 64:]        # U12 = L11^-1 A12
        if n - kj < 128:
            continue  # a last outer panel of 64
        # step 1 at ki = kj + 64: its diagonal block, then rows / columns past kj + 128,
        # each first minus the product with step 0's L and U
        ki = kj + 64
        a[ki:ki + 64, ki:ki + 64] -= a[ki:ki + 64, kj:ki] @ a[kj:ki, ki:ki + 64]
        ui, li = diag_step(a, ki)
        rows = a[ki + 64:, ki:ki + 64] - a[ki + 64:, kj:ki] @ a[kj:ki, ki:ki + 64]
        a[ki + 64:, ki:ki + 64] = rows @ ui
        cols = a[ki:ki + 64, ki + 64:] - a[ki:ki + 64, kj:ki] @ a[kj:ki, ki + 64:]
        a[ki:ki + 64, ki + 64:] = li @ cols
    return a


@pytest.mark.parametrize("n", [64, 128, 192, 320, 384, 448])
def test_left_looking_schedule_equals_plain_lu(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n)) + n * np.eye(n)  # diagonally dominant: no pivoting needed
    ref = plain_lu(a)
    got = schedule_lu(a)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    lo = np.tril(got, -1) + np.eye(n)
    assert np.max(np.abs(lo @ np.triu(got) - a)) <= 1e-10 * np.max(np.abs(a))


def test_schedule_with_a_dropped_block_row_update_fails():
    """The check is sharp: a schedule that leaves out the earlier panels'
    products on a panel's block row (a plausible slip in the regions) no
    longer gives the LU."""
    n = 320
    rng = np.random.default_rng(3)
    a = rng.standard_normal((n, n)) + n * np.eye(n)
    ref = plain_lu(a)
    assert np.max(np.abs(schedule_lu(a) - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert np.max(np.abs(schedule_lu(a, drop_row_update=True) - ref)) > 1e-6 * np.max(np.abs(ref))
