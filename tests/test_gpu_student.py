"""The learned part: student forward/backward/Adam kernels vs the FP64 oracle, reproducibility and
checkpoint/resume, the gain of training, and the teacher-fallback cascade. Through the C ABI."""
import os

import numpy as np
import pytest

import oracle
import synth
from _common import TOL, infer, make_net, student_params, teacher_params

pytestmark = pytest.mark.gpu

S = synth.STUDENT
T = synth.TEACHER


def bf16_round(a):
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def lib():
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    return m


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_student_forward_matches_oracle(lib, prec):
    """FP32 student (CUDA cores) within 1e-5 of the oracle; BF16 student (BF16 weights, the fused
    tensor-core kernel with BF16 layer-1 features) within the BF16 bar."""
    m = lib
    p32 = student_params()
    net = make_net(S, {"fp32": m.MB_PREC_FP32, "bf16": m.MB_PREC_BF16}[prec], p32)
    v = synth.em_volume(3001, 2, 70, 45)
    out = infer(net, v)
    pref = bf16_round(p32) if prec == "bf16" else p32
    for zi in range(2):
        ref = oracle.forward_region(S, pref, v[zi])
        if prec == "fp32":
            assert np.abs(out[zi] - ref).max() <= 1e-5
        else:  # a 70x45 map: max-abs and mean-abs (agreement is asserted on maps >= 4096 px)
            met = oracle.metrics(out[zi], ref)
            assert met["max_abs"] <= TOL["bf16"]["max_abs"] and met["mean_abs"] <= TOL["bf16"]["mean_abs"], met
    net.close()


@pytest.mark.parametrize("prec,shape", [("fp32", (3, 40, 52)), ("bf16", (3, 40, 52)), ("fp32", (4, 100, 130))])
def test_student_gradient_matches_oracle(lib, prec, shape):
    """Loss and gradient vs the FP64 oracle; (4, 100, 130) spans many 16x16 tiles per slice, with
    ragged tiles at the bottom and right edges."""
    import torch
    m = lib
    p32 = synth.init_params(S, synth.STUDENT_WEIGHT_SEED, bias_std=0.05)
    net = make_net(S, {"fp32": m.MB_PREC_FP32, "bf16": m.MB_PREC_BF16}[prec], p32)
    v = synth.em_volume(3002, *shape)
    tgt = np.random.default_rng(3).uniform(0.05, 0.95, size=v.shape).astype(np.float32)
    grad = torch.empty(net.n_params, dtype=torch.float32, device="cuda")
    loss = m.mb_student_loss_grad(net.handle, torch.from_numpy(v).cuda(), torch.from_numpy(tgt).cuda(), *shape,
                                  grad)
    pref = bf16_round(p32) if prec == "bf16" else p32
    loss_ref, g_ref = oracle.student_loss_grad(S, pref, v, tgt)
    g = grad.cpu().numpy()
    assert abs(loss - loss_ref) <= 1e-5 * abs(loss_ref)
    rel = np.abs(g - g_ref).max() / np.abs(g_ref).max()
    assert rel <= 1e-4, rel
    net.close()


def test_adam_first_step_matches_oracle(lib):
    import torch
    m = lib
    p32 = synth.init_params(S, synth.STUDENT_WEIGHT_SEED, bias_std=0.05)
    net = make_net(S, m.MB_PREC_FP32, p32)
    v = synth.em_volume(3003, 4, 32, 32)
    tgt = np.random.default_rng(4).uniform(0.1, 0.9, size=v.shape).astype(np.float32)
    # one step on a batch of one slice: the sampled slice is known from the seeded sampler, so
    # train on 1 slice (the sampler can only pick it)
    cfg = m.train_cfg(batch=1, steps=1, lr=1e-3, seed=11)
    m.mb_student_train(net.handle, torch.from_numpy(v[:1]).cuda(), torch.from_numpy(tgt[:1]).cuda(), 1, 32, 32, cfg)
    w = np.empty(net.n_params, dtype=np.float32)
    m.mb_get_weights(net.handle, w)
    _, g_ref = oracle.student_loss_grad(S, p32, v[:1], tgt[:1])
    z = np.zeros(net.n_params)
    w_ref, _, _ = oracle.student_adam_step(S, p32.astype(np.float64), z, z, g_ref, step=1, lr=1e-3)
    assert np.abs(w - w_ref).max() <= 2e-5 * 1e-3 + 1e-7
    net.close()


def test_two_training_steps_match_oracle(lib):
    """Two updates on one slice: from step 2 the Adam moments (of the centred layer-1 gradients)
    enter the update, so this pins the moments' coordinates as well as the step."""
    import torch
    m = lib
    p32 = synth.init_params(S, synth.STUDENT_WEIGHT_SEED, bias_std=0.05, centred_input=True)
    net = make_net(S, m.MB_PREC_FP32, p32)
    v = synth.em_volume(3005, 1, 40, 36)
    tgt = np.random.default_rng(5).uniform(0.1, 0.9, size=v.shape).astype(np.float32)
    cfg = m.train_cfg(batch=1, steps=2, lr=1e-3, seed=13)
    m.mb_student_train(net.handle, torch.from_numpy(v).cuda(), torch.from_numpy(tgt).cuda(), 1, 40, 36, cfg)
    w = np.empty(net.n_params, dtype=np.float32)
    m.mb_get_weights(net.handle, w)
    wr = p32.astype(np.float64)
    mo = np.zeros(net.n_params)
    vo = np.zeros(net.n_params)
    for step in (1, 2):
        # the FP32 GPU forward uses the FP32 weights, so the oracle takes them unrounded
        _, g = oracle.student_loss_grad(S, wr.astype(np.float32), v, tgt)
        if step == 1:
            g1 = np.abs(oracle.centred_grad(S, g))
        wr, mo, vo = oracle.student_adam_step(S, wr, mo, vo, g, step=step, lr=1e-3)
    # The first step moves a parameter by about lr * sign(g): where the centred gradient is within
    # the GPU gradient's tolerance (1e-4 of the largest) of zero its sign is not determined, and the
    # parameter may legitimately land up to 2 lr per step away. Everywhere else: tight.
    sure = g1 > 1e-3 * g1.max()
    err = np.abs(w - wr)
    assert err[sure].max() <= 2 * (2e-5 * 1e-3) + 2e-7, err[sure].max()
    assert err.max() <= 4e-3 + 1e-6
    assert sure.sum() >= 0.8 * net.n_params * (g1 > 0).mean()
    net.close()


def _train(m, prec, v, tgt, steps, seed, ckpt=None, ckpt_every=0, resume=0, batch=4, params=None):
    import torch
    net = make_net(S, prec, student_params() if params is None else params)
    cfg = m.train_cfg(batch=batch, steps=steps, ckpt_every=ckpt_every, resume=resume, lr=1e-3, seed=seed)
    curve = np.zeros(steps, dtype=np.float32)
    z, h, w = v.shape
    m.mb_student_train(net.handle, torch.from_numpy(v).cuda(), torch.from_numpy(tgt).cuda(), z, h, w, cfg, ckpt,
                       curve)
    wts = np.empty(net.n_params, dtype=np.float32)
    m.mb_get_weights(net.handle, wts)
    return net, wts, curve


@pytest.fixture(scope="module")
def small_data(lib):
    import torch
    m = lib
    v = synth.em_volume(3100, 12, 64, 64)
    teacher = make_net(T, m.MB_PREC_FP32, teacher_params())
    tgt = infer(teacher, v)
    teacher.close()
    return v, tgt


def test_training_is_bitwise_reproducible(lib, small_data):
    m = lib
    v, tgt = small_data
    n1, w1, c1 = _train(m, m.MB_PREC_BF16, v, tgt, 12, seed=5)
    n2, w2, c2 = _train(m, m.MB_PREC_BF16, v, tgt, 12, seed=5)
    np.testing.assert_array_equal(w1, w2)
    np.testing.assert_array_equal(c1, c2)
    n1.close()
    n2.close()


def test_resume_from_checkpoint_is_bitwise_identical(lib, small_data, tmp_path):
    m = lib
    v, tgt = small_data
    full_net, w_full, c_full = _train(m, m.MB_PREC_BF16, v, tgt, 20, seed=6)
    ck = str(tmp_path / "student.ckpt")
    # a run that stops after 10 steps (checkpoint at step 10), then a fresh process-like resume
    part, _, _ = _train(m, m.MB_PREC_BF16, v, tgt, 10, seed=6, ckpt=ck, ckpt_every=10)
    assert os.path.exists(ck)
    res, w_res, c_res = _train(m, m.MB_PREC_BF16, v, tgt, 20, seed=6, ckpt=ck, ckpt_every=10, resume=1)
    np.testing.assert_array_equal(w_res, w_full)
    np.testing.assert_array_equal(c_res[:10], c_full[10:])
    for n in (full_net, part, res):
        n.close()


def test_resume_rejects_a_checkpoint_of_another_format(lib, small_data, tmp_path):
    """A file at the checkpoint path that is not a format-2 checkpoint of this student (an older
    version, or a truncated file) is an error, and the file is left as it was."""
    m = lib
    v, tgt = small_data
    import struct
    for name, blob in (("v1.ckpt", b"MBCKPT01" + struct.pack("<qqqq", 10, 0, 6, 0) + bytes(64)),
                       ("short.ckpt", b"MBCKPT02" + bytes(40))):
        ck = tmp_path / name
        ck.write_bytes(blob)
        with pytest.raises(m.MembraneError) as e:
            _train(m, m.MB_PREC_BF16, v, tgt, 4, seed=6, ckpt=str(ck), ckpt_every=2, resume=1)
        assert e.value.status == m.MB_ERR_INVALID_ARG
        assert ck.read_bytes() == blob
    # without resume, or with no file at the path, training starts fresh
    fresh = tmp_path / "absent.ckpt"
    net, _, _ = _train(m, m.MB_PREC_BF16, v, tgt, 2, seed=6, ckpt=str(fresh), ckpt_every=2, resume=1)
    assert fresh.exists()
    net.close()


def test_training_gains_over_untrained_student(lib, small_data):
    """What the trained network gains: its error against the teacher drops well below the
    untrained student's, on held-out slices."""
    m = lib
    v, tgt = small_data
    net, _, curve = _train(m, m.MB_PREC_BF16, v[:10], tgt[:10], 150, seed=7, batch=4)
    held = v[10:]
    ref = tgt[10:]
    trained = infer(net, held)
    untrained_net = make_net(S, m.MB_PREC_BF16, student_params())
    untrained = infer(untrained_net, held)
    e_tr = np.abs(trained - ref).mean()
    e_un = np.abs(untrained - ref).mean()
    assert curve[-10:].mean() < 0.5 * curve[:10].mean()
    assert e_tr < 0.5 * e_un, (e_tr, e_un)
    net.close()
    untrained_net.close()


def _tile_fracs(sp, tile, lo, hi):
    z, h, w = sp.shape
    nty, ntx = (h + tile - 1) // tile, (w + tile - 1) // tile
    cnt = np.zeros((z, nty, ntx), dtype=np.int64)
    size = np.zeros((nty, ntx), dtype=np.int64)
    for ty in range(nty):
        for tx in range(ntx):
            blk = sp[:, ty * tile:min(h, ty * tile + tile), tx * tile:min(w, tx * tile + tile)]
            cnt[:, ty, tx] = ((blk >= lo) & (blk <= hi)).reshape(z, -1).sum(axis=1)
            size[ty, tx] = blk.shape[1] * blk.shape[2]
    return cnt, size


@pytest.mark.parametrize("tprec", ["bf16", "fp32"])
def test_cascade_fallback_tiles_equal_teacher(lib, small_data, tprec):
    """Flagged tiles carry the teacher's output bitwise, the others the student's; the flag is the
    stated rule applied to the student's own map. The band and threshold are chosen from the
    student's output so both kinds of tile occur (the stand-in teacher's maps sit near 0.58)."""
    import torch
    m = lib
    v, tgt = small_data
    student, _, _ = _train(m, m.MB_PREC_BF16, v[:10], tgt[:10], 40, seed=8)
    teacher = make_net(T, {"bf16": m.MB_PREC_BF16, "fp32": m.MB_PREC_FP32}[tprec], teacher_params())
    vol = synth.em_volume(3200, 3, 96, 80)
    s_only = infer(student, vol)
    t_only = infer(teacher, vol)
    tile = 32
    lo, hi = np.float32(np.quantile(s_only, 0.45)), np.float32(np.quantile(s_only, 0.55))
    cnt, size = _tile_fracs(s_only, tile, lo, hi)
    max_frac = np.float32(np.median(cnt / size))
    expect = cnt.astype(np.float64) > np.float64(max_frac) * size
    assert expect.any() and not expect.all()
    x = torch.from_numpy(vol).cuda()
    out = torch.empty((3, 96, 80), dtype=torch.float32, device="cuda")
    flags = torch.zeros(expect.size, dtype=torch.uint8, device="cuda")
    rate = m.mb_infer_cascade(student.handle, teacher.handle, x, 3, 96, 80, out, tile, float(lo), float(hi),
                              float(max_frac), flags)
    out = out.cpu().numpy()
    flags = flags.cpu().numpy().reshape(expect.shape).astype(bool)
    np.testing.assert_array_equal(flags, expect)
    assert abs(rate - expect.mean()) < 1e-12
    for zi in range(3):
        for ty in range(expect.shape[1]):
            for tx in range(expect.shape[2]):
                ys, xs = slice(ty * tile, min(96, ty * tile + tile)), slice(tx * tile, min(80, tx * tile + tile))
                want = t_only[zi, ys, xs] if expect[zi, ty, tx] else s_only[zi, ys, xs]
                np.testing.assert_array_equal(out[zi, ys, xs], want)
    student.close()
    teacher.close()


def test_cascade_with_the_stated_band(lib, small_data):
    """The stated rule (256x256 tiles, [0.3, 0.7], 5%): the rate equals the rule's prediction."""
    import torch
    m = lib
    v, tgt = small_data
    student, _, _ = _train(m, m.MB_PREC_BF16, v[:10], tgt[:10], 20, seed=9)
    teacher = make_net(T, m.MB_PREC_BF16, teacher_params())
    vol = synth.em_volume(3201, 2, 300, 280)
    s_only = infer(student, vol)
    cnt, size = _tile_fracs(s_only, 256, np.float32(0.3), np.float32(0.7))
    expect = cnt.astype(np.float64) > np.float64(np.float32(0.05)) * size
    x = torch.from_numpy(vol).cuda()
    out = torch.empty((2, 300, 280), dtype=torch.float32, device="cuda")
    rate = m.mb_infer_cascade(student.handle, teacher.handle, x, 2, 300, 280, out, 256, 0.3, 0.7, 0.05)
    assert abs(rate - expect.mean()) < 1e-12
    if expect.all():
        np.testing.assert_array_equal(out.cpu().numpy(), infer(teacher, vol))
    student.close()
    teacher.close()
