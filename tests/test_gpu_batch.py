"""Batching of independent uneven blocks (Sec. 2: blocks are segmented independently): one
persistent launch per batch under a captured CUDA graph equals per-block inference bitwise; the
autotuner's choice changes no result. Through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from _common import TOL, infer, make_net, teacher_params

pytestmark = pytest.mark.gpu

T = synth.TEACHER


def make_blocks(shapes, seed, pitch_pad=0):
    import torch
    vols, ins, outs, blocks = [], [], [], []
    for i, (d, h, w) in enumerate(shapes):
        v = synth.em_volume(seed, d, h, w, block=i)
        vols.append(v)
        wp = w + pitch_pad
        x = torch.zeros((d, h, wp), dtype=torch.uint8, device="cuda")
        x[:, :, :w] = torch.from_numpy(v).cuda()
        o = torch.full((d, h, wp), -1.0, dtype=torch.float32, device="cuda")
        ins.append(x)
        outs.append(o)
        blocks.append((x, d, h, w, wp, h * wp, o, wp, h * wp))
    return vols, ins, outs, blocks


@pytest.fixture(scope="module")
def bf16():
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    n = make_net(T, m.MB_PREC_BF16, teacher_params())
    yield n
    n.close()


def test_batch_equals_per_block_and_volume(bf16):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    shapes = [(2, 37, 300), (1, 256, 129), (3, 64, 64), (1, 8, 8), (2, 120, 250), (1, 300, 40)]
    vols, ins, outs, blocks = make_blocks(shapes, 4001, pitch_pad=5)
    m.mb_infer_batch(bf16.handle, blocks)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(-1.0)
    m.mb_infer_batch(bf16.handle, blocks)  # graph replay
    torch.cuda.synchronize()
    for a, b in zip(first, outs):
        assert torch.equal(a, b)
    _, _, outs_pb, blocks_pb = make_blocks(shapes, 4001, pitch_pad=5)
    m.mb_infer_batch_per_block(bf16.handle, blocks_pb)
    torch.cuda.synchronize()
    for (d, h, w), v, a, b in zip(shapes, vols, outs, outs_pb):
        assert torch.equal(a[:, :, :w], b[:, :, :w])
        assert bool((a[:, :, w:] == -1.0).all())          # pitch padding untouched
        np.testing.assert_array_equal(a[:, :, :w].cpu().numpy(), infer(bf16, v))
    ref = oracle.forward_region(T, teacher_params(), vols[1][0])
    assert oracle.metrics(outs[1][0, :, :129].cpu().numpy(), ref)["max_abs"] <= TOL["bf16"]["max_abs"]


def test_batch_more_blocks_than_one_launch_holds(bf16):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    rng = np.random.default_rng(9)
    shapes = [(int(rng.integers(1, 3)), int(rng.integers(8, 40)), int(rng.integers(8, 40))) for _ in range(70)]
    vols, ins, outs, blocks = make_blocks(shapes, 4002)
    m.mb_infer_batch(bf16.handle, blocks)
    torch.cuda.synchronize()
    for v, o in zip(vols, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), infer(bf16, v))


def test_autotune_choice_and_cache(bf16, tmp_path):
    from paper_1612_02120_gb300 import membrane as m
    v = synth.em_volume(4003, 2, 300, 260)
    before = infer(bf16, v)
    cache = str(tmp_path / "tune.json")
    c1 = m.mb_autotune(bf16.handle, 2, 300, 260, cache)
    assert not c1["from_cache"] and c1["rows_per_item"] in (0, 64, 128, 256, 512, 1024) and c1["stages"] in (4, 5, 6)
    c2 = m.mb_autotune(bf16.handle, 2, 300, 260, cache)
    assert c2["from_cache"] and c2["rows_per_item"] == c1["rows_per_item"] and c2["stages"] == c1["stages"]
    np.testing.assert_array_equal(infer(bf16, v), before)


def test_batch_autotune_on_the_batch_itself(bf16, tmp_path):
    """The batch tuner times every candidate on the caller's blocks: its choice is a candidate, it is
    cached under the blocks' shapes (other addresses, same shapes: a hit), the outputs it leaves are
    the batch's maps, and the batch maps the same afterwards."""
    import torch
    from paper_1612_02120_gb300 import membrane as m
    shapes = [(2, 37, 300), (1, 256, 129), (3, 64, 64)]
    vols, _, outs, blocks = make_blocks(shapes, 4012)
    m.mb_set_tuning(bf16.handle, 1024, 6)
    m.mb_infer_batch(bf16.handle, blocks)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    for o in outs:
        o.fill_(-1.0)
    cache = str(tmp_path / "tune.json")
    c1 = m.mb_autotune_batch(bf16.handle, blocks, m.MB_OUT_F32, cache)
    assert not c1["from_cache"] and c1["rows_per_item"] in (0, 64, 128, 256, 512, 1024) and c1["stages"] in (4, 5, 6)
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
    _, _, outs2, blocks2 = make_blocks(shapes, 4012)
    c2 = m.mb_autotune_batch(bf16.handle, blocks2, m.MB_OUT_F32, cache)
    assert c2["from_cache"] and (c2["rows_per_item"], c2["stages"]) == (c1["rows_per_item"], c1["stages"])
    m.mb_infer_batch(bf16.handle, blocks2)
    torch.cuda.synchronize()
    for a, b in zip(outs2, ref):
        assert torch.equal(a, b)
    lib = m.load()
    assert lib.mb_autotune_batch(bf16.handle, None, 0, 0, None, None, None) == m.MB_ERR_INVALID_ARG
    m.mb_set_tuning(bf16.handle, 1024, 6)


def test_fp32_batch_uses_per_block_path():
    import torch
    from paper_1612_02120_gb300 import membrane as m
    net = make_net(T, m.MB_PREC_FP32, teacher_params())
    shapes = [(1, 30, 20), (2, 16, 45)]
    vols, ins, outs, blocks = make_blocks(shapes, 4004)
    m.mb_infer_batch(net.handle, blocks)
    torch.cuda.synchronize()
    for v, o in zip(vols, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), infer(net, v))
    net.close()


def test_every_tuning_candidate_gives_the_same_maps(bf16):
    """The autotuner's knobs (rows per work item or the even-range split, A-ring depth) change the
    schedule, never a value: every BF16 candidate, applied with mb_set_tuning, maps a volume and an
    uneven batch bitwise as the default does."""
    import torch
    from paper_1612_02120_gb300 import membrane as m
    v = synth.em_volume(4010, 3, 300, 260)
    shapes = [(2, 37, 300), (1, 256, 129), (3, 64, 64)]
    vols, _, outs, blocks = make_blocks(shapes, 4011)
    m.mb_set_tuning(bf16.handle, 1024, 6)
    ref = infer(bf16, v)
    m.mb_infer_batch(bf16.handle, blocks)
    torch.cuda.synchronize()
    ref_b = [o.clone() for o in outs]
    for rows in (64, 128, 256, 512, 1024, 0):
        for stages in (4, 5, 6):
            m.mb_set_tuning(bf16.handle, rows, stages)
            np.testing.assert_array_equal(infer(bf16, v), ref, err_msg=f"rows {rows} stages {stages}")
            for o in outs:
                o.fill_(-1.0)
            m.mb_infer_batch(bf16.handle, blocks)
            torch.cuda.synchronize()
            for a, b in zip(outs, ref_b):
                assert torch.equal(a, b), (rows, stages)
    m.mb_set_tuning(bf16.handle, 1024, 6)


def test_fp8_tuning_candidates_and_cache(tmp_path):
    """FP8 nets tune the ring depth only (rows per item reported as 0); every depth gives the same
    maps; the choice is cached; invalid choices are rejected."""
    import torch
    from paper_1612_02120_gb300 import membrane as m
    net = make_net(T, m.MB_PREC_FP8, teacher_params())
    cal = torch.from_numpy(synth.em_volume(synth.BASE_SEED + 3, 4, 256, 256)).cuda()
    m.mb_calibrate_fp8(net.handle, cal, 4, 256, 256)
    v = synth.em_volume(4012, 3, 200, 300)
    ref = infer(net, v)
    for stages in (4, 6, 8):
        m.mb_set_tuning(net.handle, 0, stages)
        np.testing.assert_array_equal(infer(net, v), ref, err_msg=f"stages {stages}")
    cache = str(tmp_path / "tune.json")
    c1 = m.mb_autotune(net.handle, 2, 300, 260, cache)
    assert not c1["from_cache"] and c1["rows_per_item"] == 0 and c1["stages"] in (4, 6, 8)
    c2 = m.mb_autotune(net.handle, 2, 300, 260, cache)
    assert c2["from_cache"] and c2["stages"] == c1["stages"]
    lib = m.load()
    assert lib.mb_set_tuning(net.handle, 0, 5) == m.MB_ERR_INVALID_ARG      # not a compiled FP8 depth
    assert lib.mb_set_tuning(net.handle, 64, 6) == m.MB_ERR_INVALID_ARG     # FP8 has no item length
    net.close()


def test_set_tuning_rejects_what_it_cannot_apply(bf16):
    from paper_1612_02120_gb300 import membrane as m
    lib = m.load()
    assert lib.mb_set_tuning(bf16.handle, 96, 6) == m.MB_ERR_INVALID_ARG
    assert lib.mb_set_tuning(bf16.handle, 256, 8) == m.MB_ERR_INVALID_ARG
    assert lib.mb_set_tuning(None, 256, 6) == m.MB_ERR_INVALID_ARG
    fp32 = make_net(T, m.MB_PREC_FP32, teacher_params())
    assert lib.mb_set_tuning(fp32.handle, 256, 6) == m.MB_ERR_UNSUPPORTED
    fp32.close()
