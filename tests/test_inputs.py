"""The seeded input generator: host statistics, and device/host agreement (GPU)."""
import numpy as np
import pytest

import hessgen


def test_isotropic_covariance():
    h = hessgen.hessian_planes(2511, 0, 0, 2.0, 200000)
    cov = np.cov(h) / 4.0 * 15.0  # s = 2
    want = np.zeros((6, 6))
    want[:3, :3] = 1.0
    want[np.arange(3), np.arange(3)] = 3.0
    want[np.arange(3, 6), np.arange(3, 6)] = 1.0
    np.testing.assert_allclose(cov, want, atol=0.05)
    assert abs(np.var(h[:3].sum(0)) / 4.0 - 1.0) < 0.02  # var(tr) = s^2


def test_streams_are_independent_and_reproducible():
    a = hessgen.hessian_planes(1, 0, 0, 1.0, 1000)
    b = hessgen.hessian_planes(1, 0, 0, 1.0, 1000)
    c = hessgen.hessian_planes(1, 0, 1, 1.0, 1000)
    d = hessgen.hessian_planes(1, 1, 0, 1.0, 1000)
    assert np.array_equal(a, b)
    assert not np.allclose(a, c) and not np.allclose(a, d)
    sub = hessgen.hessian_points(1, 0, 0, 1.0, np.array([5, 999, 17]))
    np.testing.assert_array_equal(sub, a[:, [5, 999, 17]])


def test_philox_known_answers():
    """Known-answer vectors of Philox-4x32-10 (Salmon et al. 2011)."""
    cases = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in cases:
        got = hessgen.philox4x32_10(np.array(ctr, dtype=np.uint32)[:, None], np.array(key, dtype=np.uint32))
        assert [int(x) for x in got[:, 0]] == want


@pytest.mark.gpu
def test_device_generator_matches_host():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import hessgen.device as hdev
    hdev.build()
    n = 100003
    for dt, npdt in ((torch.float64, np.float64), (torch.float32, np.float32)):
        buf = torch.empty((6, n + 5), dtype=dt, device="cuda")
        hdev.fill(buf[:, :n], 2512, 3, 7, 1.7, point_offset=12345)
        torch.cuda.synchronize()
        got = buf[:, :n].cpu().numpy()
        want = hessgen.hessian_points(2512, 3, 7, 1.7, np.arange(12345, 12345 + n), dtype=npdt)
        diff = np.abs(got.astype(np.float64) - want.astype(np.float64))
        if npdt == np.float64:
            # ulp-level differences of the Box-Muller transcendentals, on the scale s
            assert diff.max() <= 1e-14 * 1.7
        else:
            # at most one FP32 rounding step apart
            assert np.all(diff <= np.spacing(np.abs(want)).astype(np.float64) * 1.0001)
        assert (got == want).mean() > 0.5  # most values are bit-identical
