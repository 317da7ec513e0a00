"""Dynamic channel swapping (Section 2): images ranked by PSNR go to the
wavelengths from the longest down."""
import numpy as np

from oracle import dos_oracle as O
from paper_2604_02624_gb300.design import channel_swap


def test_best_image_goes_to_longest_wavelength():
    lam = np.array([500, 740, 620, 560]) * 1e-9
    psnr = np.array([30.0, 10.0, 45.0, 20.0])
    perm = channel_swap(psnr, lam)
    assert perm[1] == 2          # longest (740) gets the best image (45 dB)
    assert perm[2] == 0          # next (620) gets 30 dB
    assert perm[3] == 3          # 560 gets 20 dB
    assert perm[0] == 1          # shortest gets the hardest image


def test_swap_is_a_permutation_and_ordered():
    rng = np.random.default_rng(2)
    lam = np.linspace(750e-9, 450e-9, 4096)[rng.permutation(4096)]
    psnr = rng.normal(45, 2, 4096)
    perm = channel_swap(psnr, lam)
    assert np.array_equal(np.sort(perm), np.arange(4096))
    new_psnr = psnr[perm]
    order = np.argsort(-lam)
    assert np.all(np.diff(new_psnr[order]) <= 0)


def test_ties_keep_the_original_order():
    lam = np.array([700.0, 600.0, 500.0])
    perm = channel_swap(np.array([5.0, 5.0, 5.0]), lam)
    assert np.array_equal(perm, [0, 1, 2])


def test_oracle_swap_hand_case():
    """Four channels: the 740 nm channel takes the 45 dB image, 620 nm the
    30 dB one, 560 nm the 20 dB one and 500 nm the 10 dB one."""
    lam = np.array([500, 740, 620, 560]) * 1e-9
    psnr = np.array([30.0, 10.0, 45.0, 20.0])
    assert O.channel_swap(psnr, lam).tolist() == [1, 2, 0, 3]


def test_oracle_swap_is_a_sorted_assignment():
    """After the swap the PSNR of the assigned image never increases as the
    wavelength decreases, and every image is used once."""
    rng = np.random.default_rng(3)
    lam = np.linspace(750e-9, 450e-9, 257)[rng.permutation(257)]
    psnr = np.round(rng.normal(45, 2, 257), 1)   # with ties
    perm = O.channel_swap(psnr, lam)
    assert sorted(perm.tolist()) == list(range(257))
    by_lambda = psnr[perm][np.argsort(-lam, kind="stable")]
    assert np.all(np.diff(by_lambda) <= 0)
