"""The continuous-batching server (cvc_server_*): every result must be the
same alone and in a mix of concurrent streams (bit-identical to a plain
codec fed the same requests), sessions are admitted by device memory, and a
session's requests run in order.
"""
import time

import numpy as np
import pytest
import torch

from paper_1510_00561_b300 import Batch, Codec, CvcError, Server
from paper_1510_00561_b300 import synthetic as S

pytestmark = pytest.mark.gpu

QCIF = dict(width=176, height=144, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=4)
CIF = dict(width=352, height=288, levels=3, dirs_log2=[3, 2, 2], qph=8, qpl=1, key_interval=4)
VGA = dict(width=640, height=480, levels=4, dirs_log2=[4, 3, 3, 2], qph=8, qpl=1, key_interval=4)
ODD = dict(width=101, height=77, levels=2, dirs_log2=[2, 2], qph=16, qpl=2, key_interval=3)

_frames = {}


def _video(cfg, seed, n):
    key = (cfg["width"], cfg["height"], seed, n)
    if key not in _frames:
        v = S.SyntheticVideo(S.spec_for(cfg["width"], cfg["height"], seed=seed))
        _frames[key] = [torch.from_numpy(f).cuda() for f in v.frames(n)]
    return _frames[key]


def _drain(server, want, timeout_s=60.0):
    got = []
    t0 = time.time()
    while len(got) < want:
        got += server.poll(wait_us=2000)
        assert time.time() - t0 < timeout_s, "server did not complete %d requests" % want
    return got


class _Req:
    """Buffers of one encode+decode request, kept until its completion is checked."""

    def __init__(self, cfg, frame, max_stream):
        self.frame = frame
        self.out = torch.empty(max_stream, dtype=torch.uint8, device="cuda")
        self.rgb = torch.empty((cfg["height"], cfg["width"], 3), dtype=torch.uint8, device="cuda")


def _max_stream(cfg):
    return Codec(**cfg).max_stream


def _plain_results(cfg, frames):
    c = Codec(**cfg)
    d = Codec(**cfg)
    out = []
    for f in frames:
        s, ft = c.encode(f)
        out.append((s.clone(), d.decode(s.clone()).clone(), ft))
    return out


def _serve(mix, order_seed, budget=64 << 30, slots=4, depth=1):
    """Run sessions `mix` = [(cfg, frames)] through one server, submitting
    their frames interleaved in a seeded random order (each session's frames
    in order) with polls in between; returns per session [(bytes, rgb, type)]."""
    srv = Server(budget, slots_per_shard=slots, steps_in_flight=depth)
    sids = [srv.open(**cfg) for cfg, _ in mix]
    ms = [_max_stream(cfg) for cfg, _ in mix]
    rng = np.random.default_rng(order_seed)
    pending = [list(range(len(fr))) for _, fr in mix]
    reqs = {}
    results = [[None] * len(fr) for _, fr in mix]
    tag = 0
    n_sub = 0
    while any(pending):
        live = [i for i in range(len(mix)) if pending[i]]
        i = int(rng.choice(live))
        t = pending[i].pop(0)
        cfg, fr = mix[i]
        r = _Req(cfg, fr[t], ms[i])
        reqs[tag] = (i, t, r)
        srv.submit(sids[i], 3, rgb=r.frame, out=r.out, rgb_out=r.rgb, tag=tag)
        tag += 1
        n_sub += 1
        if rng.random() < 0.5:
            for c in srv.poll(wait_us=int(rng.integers(0, 300))):
                _take(c, reqs, results)
    for c in _drain(srv, n_sub - sum(x is not None for res in results for x in res)):
        _take(c, reqs, results)
    st = srv.stats()
    assert st["requests_queued"] == 0
    return results, st


def _take(c, reqs, results):
    i, t, r = reqs.pop(c["tag"])
    assert c["enc_status"] == 0 and c["dec_status"] == 0, c
    results[i][t] = (r.out[:c["out_len"]].clone(), r.rgb.clone(), c["frame_type"])
    assert c["t_submit_ns"] <= c["t_launch_ns"] <= c["t_done_ns"]


def _same(a, b):
    assert len(a) == len(b)
    for (s1, r1, t1), (s2, r2, t2) in zip(a, b):
        assert t1 == t2 and torch.equal(s1, s2) and torch.equal(r1, r2)


def test_results_are_the_same_alone_and_in_a_mix():
    target = (QCIF, _video(QCIF, 1, 6))
    alone = _serve([target], 0)[0][0]
    _same(alone, _plain_results(*target))
    mix = [target] + [(cfg, _video(cfg, 10 + j, 5)) for j, cfg in
                      enumerate([QCIF, CIF, VGA, ODD, QCIF, CIF, ODD, QCIF, VGA, QCIF, CIF])]
    for seed, depth in ((1, 1), (2, 1), (3, 2), (4, 3)):
        # with several steps in flight per shard, partly filled steps skip their idle slots
        res, st = _serve(mix, seed, depth=depth)
        _same(res[0], alone)
        assert st["shards"] >= 4 and st["peak_used_bytes"] <= st["budget_bytes"]
    for (cfg, fr), r in zip(mix[1:4], res[1:4]):
        _same(r, _plain_results(cfg, fr))


def test_admission_by_memory_budget():
    budget = Batch.device_bytes([QCIF])       # exactly one one-slot QCIF shard
    srv = Server(budget, slots_per_shard=1)
    ids = [srv.open(**QCIF) for _ in range(3)]
    st = srv.stats()
    assert st["active_sessions"] == 1 and st["waiting_sessions"] == 2 and st["used_bytes"] <= budget
    frames = [_video(QCIF, 20 + i, 2) for i in range(3)]
    ms = _max_stream(QCIF)
    reqs, results = {}, [[None] * 2 for _ in range(3)]
    tag = 0
    for i in range(3):
        for t in range(2):
            r = _Req(QCIF, frames[i][t], ms)
            reqs[tag] = (i, t, r)
            srv.submit(ids[i], 3, rgb=r.frame, out=r.out, rgb_out=r.rgb, tag=tag)
            tag += 1
    # only the admitted session progresses; the others wait for memory
    for c in _drain(srv, 2):
        _take(c, reqs, results)
    assert results[0][1] is not None and results[1][0] is None
    srv.poll(wait_us=1000)
    assert srv.stats()["waiting_sessions"] == 2
    srv.close(ids[0])          # frees its shard, which admits the next session
    for c in _drain(srv, 2):
        _take(c, reqs, results)
    srv.close(ids[1])
    for c in _drain(srv, 2):
        _take(c, reqs, results)
    st = srv.stats()
    assert st["peak_used_bytes"] <= budget and st["requests_done"] == 6
    for i in range(3):
        _same(results[i], _plain_results(QCIF, frames[i]))
    # a session that can never fit the budget is refused outright
    with pytest.raises(CvcError) as e:
        srv.open(**VGA)
    assert e.value.status == 8


def test_decode_requests_and_validation():
    srv = Server(8 << 30, slots_per_shard=2)
    enc = srv.open(**CIF)
    dec = srv.open(**CIF)
    frames = _video(CIF, 30, 4)
    ms = _max_stream(CIF)
    outs = [torch.empty(ms, dtype=torch.uint8, device="cuda") for _ in frames]
    for t, f in enumerate(frames):
        srv.submit(enc, 1, rgb=f, out=outs[t], tag=t)
    got = sorted(_drain(srv, 4), key=lambda c: c["tag"])
    streams = [outs[c["tag"]][:c["out_len"]].clone() for c in got]
    assert [c["frame_type"] for c in got] == [0, 1, 1, 1]
    rgbs = [torch.empty((288, 352, 3), dtype=torch.uint8, device="cuda") for _ in frames]
    for t, s in enumerate(streams):
        srv.submit(dec, 2, stream_in=s, rgb_out=rgbs[t], tag=100 + t)
    got = _drain(srv, 4)
    assert all(c["dec_status"] == 0 for c in got)
    ref = _plain_results(CIF, frames)
    for t in range(4):
        assert torch.equal(streams[t], ref[t][0]) and torch.equal(rgbs[t], ref[t][1])
    # invalid requests are refused before anything is queued
    with pytest.raises(CvcError):
        srv.submit(enc, 1, rgb=torch.empty((288, 100, 3), dtype=torch.uint8, device="cuda"), out=outs[0], tag=9)
    with pytest.raises(CvcError):
        srv.submit(enc, 3, rgb=frames[0], out=outs[0], tag=9)       # no decoder output buffer
    srv.close(enc)
    with pytest.raises(CvcError):
        srv.submit(enc, 1, rgb=frames[0], out=outs[0], tag=9)
    assert srv.stats()["requests_queued"] == 0
