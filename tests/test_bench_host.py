"""Host logic of the benchmark that needs no GPU: the oracle results the
served record checks every request against (sums over 50,000-streamline
blocks of a pool subject) and the traffic figure's scaling."""
import numpy as np

import bench
import oracle
import synth


def test_served_expected_prefixes_equal_the_oracle():
    vols, tr = synth.make_subject(4, subject=1, n_streamlines=150_000)
    pre = bench.served_expected([(vols, tr)], 50_000, 4)[0]
    assert pre.shape == (4, 2, vols.n_roi, vols.n_targets)
    assert not pre[0].any()
    for k in (1, 3):
        n = 50_000 * k
        off = tr.offsets[: n + 1]
        C, Ce, _ = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets,
                                       tr.xyz[: off[-1]], off)
        np.testing.assert_array_equal(pre[k, 0], C)
        np.testing.assert_array_equal(pre[k, 1], Ce)


def test_prefilter_traffic_scales_with_vertices_or_is_withheld():
    b, note = bench.prefilter_traffic(bench.PREFILTER_TRAFFIC["vertices"])
    if b is None:
        assert "changed" in note  # the prefilter's sources differ from the captured ones
        return
    assert b == bench.PREFILTER_TRAFFIC["bytes"]
    b2, note2 = bench.prefilter_traffic(2 * bench.PREFILTER_TRAFFIC["vertices"])
    assert b2 == 2 * b and "scaled" in note2


def test_digest_is_of_the_int32_bytes():
    a = np.arange(12, dtype=np.int64).reshape(3, 4)
    assert bench._digest(a) == bench._digest(a.astype(np.int32))
    assert bench._digest(a) != bench._digest(a + 1)
