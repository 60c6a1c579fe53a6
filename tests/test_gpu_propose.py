"""The learned proposer end to end on the GPU: it is trained by the library's
own kernels on seeded segments (bursts of random DM, width, S/N and direction
plus narrowband interference in 10 % of segments), its threshold is set on a
calibration split so that it keeps >= 96 % of the bursts the full DM grid
detects (candidates of chirp_detect: local S/N maxima >= 7), and on held-out segments it (a) keeps >= 93 % of the full-grid
detections, (b) selects under 35 % of the (DM, dump) cells, and (c) the
selective coherent search over those cells takes no more than the full grid's
wall time at this small size (within a 25 % margin for its extra launches) and
reproduces the full grid's outputs there.  Recall is measured against the
full grid's detections.  (The
bursts it still misses sit at the coherent detection limit, where the
antenna-incoherent power the proposer reads is sqrt(M) times weaker.)"""
import time

import numpy as np
import pytest

from paper_1109_3186_gb300 import propose as pp

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")

N_TRAIN, N_CAL, N_TEST = 768, 96, 96


def _pool_segments(setup):
    # spawn-started workers, created before this process touches the GPU again
    return pp.generate(setup, range(20000, 20000 + N_TRAIN + N_CAL + N_TEST), workers=8)


def _recall(prop, segs, feats, lo, hi, thr, cache):
    s = prop.s
    found = tot = 0
    frac = []
    for i in range(lo, hi):
        dets = cache[i]
        cells = prop.cells(prop.propose(feats[i], thr), dm_margin=0)
        frac.append(cells.mean())
        for p in segs[i][1]:
            d = int(round(p.dm / (s.dms[1] - s.dms[0])))
            m = int(p.t0 // s.dump_len)
            near = [(dd, mm) for (dd, mm) in dets if abs(dd - d) <= 1 and abs(mm - m) <= 2]
            if near:
                tot += 1
                found += any(cells[dd, mm] for dd, mm in near)
    return found, tot, float(np.mean(frac))


def test_learned_proposals_keep_full_grid_detections_and_save_work():
    setup = pp.ProposalSetup()
    segs = _pool_segments(setup)
    prop = pp.Proposer(setup)
    feats = [prop.features(x) for x, _ in segs]
    ys = [pp.labels(setup, p) for _, p in segs]
    losses = prop.train(feats[:N_TRAIN], ys[:N_TRAIN], steps=1500, batch=16, lr=1e-3)
    assert np.mean(losses[-50:]) < 0.2 * losses[0]
    plan = prop.plan
    P = np.empty((setup.n_dm, plan.n_dump, plan.n_pix), np.float32)
    cache = {}
    for i in range(N_TRAIN, len(segs)):
        plan.chimageator(segs[i][0], P)
        c = plan.detect(P, 7.0)
        cache[i] = set(zip(c["dm"].tolist(), c["dump"].tolist()))
    # threshold: the highest one that keeps >= 96 % of calibration detections
    thr = None
    for t in (2.0, 1.0, 0.0, -1.0, -2.0, -3.0, -4.0, -5.0, -6.0):
        f, n, fr = _recall(prop, segs, feats, N_TRAIN, N_TRAIN + N_CAL, t, cache)
        fh, nh, frh = _recall(prop, segs, feats, N_TRAIN + N_CAL, len(segs), t, cache)
        print("threshold %.1f: calibration %d/%d (%.1f %% cells), held-out %d/%d (%.1f %% cells)"
              % (t, f, n, 100 * fr, fh, nh, 100 * frh))
        if thr is None and n and f >= 0.96 * n:
            thr = t
    assert thr is not None
    f, n, frac = _recall(prop, segs, feats, N_TRAIN + N_CAL, len(segs), thr, cache)
    print("held-out recall %d/%d at threshold %.1f, %.1f %% of cells" % (f, n, thr, 100 * frac))
    assert n > 50
    assert f >= 0.93 * n
    assert frac < 0.35
    # the selective search over the proposed cells: faster, same numbers there
    xs = [torch.from_numpy(segs[i][0]).cuda() for i in range(N_TRAIN + N_CAL, len(segs))]
    masks = [prop.cells(prop.propose(feats[i], thr), dm_margin=0)
             for i in range(N_TRAIN + N_CAL, len(segs))]
    full = torch.empty((setup.n_dm, plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
    sel = torch.empty_like(full)
    plan.chimageator(xs[0], full)
    plan.chimageator_selective(xs[0], masks[0], sel)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for x in xs:
        plan.chimageator(x, full)
    torch.cuda.synchronize()
    t_full = time.perf_counter() - t0
    t0 = time.perf_counter()
    for x, m in zip(xs, masks):
        plan.chimageator_selective(x, m, sel)
    torch.cuda.synchronize()
    t_sel = time.perf_counter() - t0
    print("full grid %.1f ms, selective %.1f ms per segment" % (1e3 * t_full / len(xs),
                                                                  1e3 * t_sel / len(xs)))
    # At this segment size (6 antennas x 2^18 samples, about 1 ms per full
    # search) the selective path's per-DM launches and its index-list upload
    # cost about as much as the transforms it skips, so the wall times are
    # compared with a margin; the work it skips is the cell fraction above,
    # and bench.py times the saving at the workload's size.
    assert t_sel < 1.25 * t_full
    plan.chimageator(xs[-1], full)
    plan.chimageator_selective(xs[-1], masks[-1], sel)
    pick = torch.from_numpy(masks[-1].astype(bool)).cuda()[:, :, None].expand_as(full)
    assert torch.equal(sel[pick], full[pick])
