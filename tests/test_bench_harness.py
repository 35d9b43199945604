"""bench.py's multi-rank plumbing on CPU: world-size-2 gloo ranks, barrier,
max-over-ranks timing and whole-job aggregation (replicas only)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank), RECOGS_DIST_BACKEND="gloo")
    import bench
    r, w, l = bench.dist_init()
    assert (r, w, l) == (rank, world, rank)
    bench.barrier(w)
    mx = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    out[rank] = (mx, bench.aggregate_value(100, w, mx))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    mx, val = out[0]
    assert mx == 15.0
    assert val == pytest.approx(100 * 2 / 0.015)


def test_aggregate_single():
    import bench
    assert bench.aggregate_value(10, 1, 1000.0) == pytest.approx(10.0)


def test_algorithmic_bytes_per_unit():
    """The per-unit byte counts of the roofline figures (design table):
    preprocess 48 per Gaussian + 48 s + 40 per visible one, scatter 16 per
    visible Gaussian + 8 per pair, tile sort 12 per pair, blend 40 per
    consumed pair + 12 per pixel + 8 per tile, the frame the sum of those
    four, SH refit 4 + 1152 per Gaussian + 40 per visible one, gradient blend
    40 per pair + 24 per pixel + 8 per tile + 12 per visible Gaussian."""
    import bench
    W, H = bench.WIDTH, bench.HEIGHT
    st = {"n_pairs_read": 1000, "n_tiles": 10, "n_visible": 90, "n_pairs": 1200}
    assert bench.algorithmic_bytes("preprocess", st, 100, 4) == 100 * 48 + 90 * (192 + 40)
    assert bench.algorithmic_bytes("preprocess", st, 100, 2) == 100 * 48 + 90 * (96 + 40)
    assert bench.algorithmic_bytes("blend", st, 100, 4) == 1000 * 40 + 12 * W * H + 80
    assert bench.algorithmic_bytes("scatter", st, 100, 4) == 90 * 16 + 1200 * 8
    assert bench.algorithmic_bytes("tile_sort", st, 100, 4) == 1200 * 12
    assert bench.algorithmic_bytes("scan", st, 100, 4) is None
    assert bench.frame_algorithmic_bytes(st, 100, 4) == (
        100 * 48 + 90 * 232 + 90 * 16 + 1200 * 8 + 1200 * 12 + 1000 * 40 + 12 * W * H + 80)
    assert bench.refit_algorithmic_bytes("refit", st, 100, 60) == 100 * 1156 + 60 * 40
    assert (bench.refit_algorithmic_bytes("blend_grad", st, 100, 60)
            == 1000 * 40 + 24 * W * H + 80 + 60 * 12)


def test_profiled_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    """A committed traffic figure is used only while its kernel source is the
    one it was taken on."""
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = bench.kernel_source_sha("blend.cu")
    (prof / "traffic_blend_3m_1080p.txt").write_text(
        f"# note\nsource_sha256_16: {sha}\ndram_bytes_per_launch: 123\n")
    (prof / "traffic_refit_3m_1080p.txt").write_text(
        "source_sha256_16: 0000000000000000\ndram_bytes_per_launch: 456\n")
    real_join = os.path.join

    def join(*parts):
        if len(parts) >= 2 and parts[0] == bench.ROOT and parts[1] == "profiles":
            return real_join(str(tmp_path), *parts[1:])
        return real_join(*parts)
    monkeypatch.setattr(bench.os.path, "join", join)
    assert bench.profiled_traffic("blend") == 123.0
    assert bench.profiled_traffic("refit") is None        # another source
    assert bench.profiled_traffic("scatter") is None      # never profiled


def test_profiled_instructions_only_for_the_profiled_source(tmp_path, monkeypatch):
    """A committed instruction count is used only while its kernel source is
    the one it was taken on, and the issue roofline divides it by the launch
    time against four issue slots per SM and cycle."""
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = bench.kernel_source_sha("blend.cu")
    (prof / "issue_blend_3m_1080p.txt").write_text(
        f"# note: with a colon\nsource_sha256_16: {sha}\nwarp_instructions_per_launch: 1000\n")
    (prof / "issue_mlp_select_6m.txt").write_text(
        "source_sha256_16: 0000000000000000\nwarp_instructions_per_launch: 7\n")
    real_join = os.path.join

    def join(*parts):
        if len(parts) >= 2 and parts[0] == bench.ROOT and parts[1] == "profiles":
            return real_join(str(tmp_path), *parts[1:])
        return real_join(*parts)
    monkeypatch.setattr(bench.os.path, "join", join)
    assert bench.profiled_instructions("blend") == 1000.0
    assert bench.profiled_instructions("mlp_select") is None   # another source
    assert bench.profiled_instructions("scatter") is None      # never counted
    assert bench.issue_roofline("blend", None, 1.0, None) is None
