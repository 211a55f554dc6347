"""Host logic of bench.py (no GPU): the traffic lookup in the committed ncu
summaries, the whole-job aggregation over ranks, and the plane sampling."""
import os

import pytest

import bench


def _write_profile(dirpath, name, digest, images, nbytes):
    os.makedirs(os.path.join(dirpath, "profiles"), exist_ok=True)
    with open(os.path.join(dirpath, "profiles", name), "w") as fh:
        fh.write(f"kernel_source_sha256_16: {digest}   (sources)\n\n"
                 f"traffic_images: {images}\ntraffic_bytes_per_launch: {nbytes}\n")


def test_traffic_is_taken_only_for_matching_sources_and_workload(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0123456789abcdef")
    _write_profile(tmp_path, "codec_u8_tma_kernel_x.md", "0123456789abcdef", 1024, 2124065280)
    assert bench.profiled_traffic(1024) == (2124065280.0, "codec_u8_tma_kernel_x.md")
    assert bench.profiled_traffic(256) == (None, None)  # another workload size
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "fedcba9876543210")
    assert bench.profiled_traffic(1024) == (None, None)  # sources changed since the capture


def test_committed_traffic_summary_is_well_formed():
    """The committed summary carries the three fields the lookup reads; when
    its hash is that of the current sources the lookup returns its bytes,
    which are within a few percent of the launch's algorithmic bytes."""
    path = os.path.join(bench.ROOT, "profiles",
                        "codec_u8_tma_kernel_batch_256x1024x1024_full.md")
    text = open(path).read()
    for key in ("kernel_source_sha256_16:", "traffic_images:", "traffic_bytes_per_launch:"):
        assert key in text
    got, _ = bench.profiled_traffic(1024)
    if got is not None:
        algo = 2 * 1024 * 1024 * 1024 + 16 * 1024
        assert 0.95 * algo < got < 1.05 * algo


class _FakeDist:
    def __init__(self, ranks_ms, ranks_blocks):
        self.ms, self.blocks = ranks_ms, ranks_blocks

    def max(self, v):
        return max(self.ms)

    def sum(self, v):
        return sum(self.blocks)


def test_aggregate_is_all_ranks_units_over_the_slowest_rank():
    d = _FakeDist([100.0, 125.0], [1000, 1000])
    value, total_ms, blocks = bench.aggregate(d, 1000, 100.0, 10)
    assert total_ms == 125.0 and blocks == 2000
    assert value == pytest.approx(2000 * 10 / 0.125)


@pytest.mark.parametrize("n,k", [(1024, 256), (1024, 1024), (10, 64), (2000, 80)])
def test_sample_indices_are_evenly_spaced_and_bounded(n, k):
    idx = bench.sample_indices(n, k)
    assert len(idx) == min(n, k)
    assert idx == sorted(set(idx)) and idx[0] == 0 and idx[-1] < n
    if k >= n:
        assert idx == list(range(n))
