"""Host-side bounds that the kernels rely on.

The uniform term of the particle form sums its mode weights per integer |n|^2 as 64-bit
integers in units of max(w) 2^-48: every mode adds at most 2^48, so a sum stays below 2^64 as
long as fewer than 2^16 modes of the stored half spectrum (Nyquist planes excluded) share one
|n|^2.  Checked here by counting at the largest grid the library accepts (512)."""
import numpy as np


def _max_modes_per_n2(n):
    h = n // 2 - 1
    f = np.arange(-h, h + 1, dtype=np.int64)
    yz = (f[:, None] ** 2 + f[None, :] ** 2).ravel()
    cnt = np.zeros(3 * h * h + 1, np.int64)
    for x in range(h + 1):  # the stored half: 0 <= n_x <= n/2 - 1
        cnt += np.bincount(x * x + yz, minlength=cnt.size)
    return int(cnt.max()), int(cnt.sum())


def test_mode_count_per_n2_fits_the_fixed_point_sums():
    for n in (16, 64, 512):
        mx, total = _max_modes_per_n2(n)
        assert total == (n // 2) * (n - 1) ** 2  # every stored non-Nyquist mode counted once
        assert mx < 2 ** 16, (n, mx)
