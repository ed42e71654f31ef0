"""Renders a fixed set of shapes through the stream, engine and allocation-free
entry points and saves every output (test helper, run as a script in a fresh
process so that MF_CHECKED selects the library before it loads):

    python tests/checked_run.py OUT.npz

Shapes: ragged frames (odd heights, widths whose last strip leaves the
frame), 1080p HEADING frames (the fast row loop), ACCEL frames whose units
no point reaches (bulk zero rows), 16-bit storage, a mixed engine tick and an
allocation-free render.  Every wait must return MF_OK: in the checked library
an access outside a plane would make it fail."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_2601_07154_gb300 as mf  # noqa: E402
from synth import StreamWorkload, WalkerSpec, hd_stream, small_stream  # noqa: E402


def main(out_path):
    dev = torch.device("cuda", 0)
    out = {}
    cases = [  # (name, width, height, window, mode, dtype)
        ("ragged333", 333, 197, 8, "heading", torch.float32),
        ("ragged257_bf16", 257, 129, 16, "heading", torch.bfloat16),
        ("w24_f16", 320, 240, 24, "accel", torch.float16),
    ]
    for name, wd, ht, win, mode, dt in cases:
        f = 0.8 * wd
        sw = StreamWorkload(name, wd, ht, 48, win, 7, (f, f, wd / 2.0, ht / 2.0),
                            WalkerSpec(n_frames=48, seed=3, turns=True, accel=1.5))
        D = torch.from_numpy(np.stack([sw.render(k) for k in range(48)])).to(dev).to(dt)
        s = mf.MotionFocusStream(wd, ht, window=win, smooth_len=7, mode=mode, device=dev,
                                 depth_dtype=dt, map_dtype=dt)
        s.push(torch.from_numpy(sw.poses).to(dev), D, sw.K())
        M, G, info, _ = s.get_maps()
        s.sync()
        out[name + "_M"] = M.float().cpu().numpy()
        out[name + "_G"] = G.float().cpu().numpy()
        out[name + "_info"] = info.view(np.uint8)
        s.close()
    for mode in ("heading", "accel"):
        w = hd_stream(n_frames=40)
        D = torch.from_numpy(np.stack([w.depth(k) for k in range(40)])).to(dev)
        s = mf.MotionFocusStream(1920, 1080, window=16, smooth_len=15, mode=mode, device=dev)
        s.push(torch.from_numpy(w.poses[:40]).to(dev), D, w.K())
        M, G, info, _ = s.get_maps()
        s.sync()
        out[f"hd_{mode}_M"] = M[16:].cpu().numpy()
        out[f"hd_{mode}_G"] = G[16:].cpu().numpy()
        s.close()
    # untuned: band heights fixed, so both libraries render the same tile geometry
    eng = mf.MotionFocusEngine(max_streams=4, max_tick_frames=64, max_stream_frames=16, device=dev,
                               tune=False)
    streams = []
    for k, (wd, ht, win) in enumerate(((640, 480, 12), (1280, 720, 24), (330, 200, 8))):
        sw = StreamWorkload(f"e{k}", wd, ht, 32, win, 7, (0.9 * wd, 0.9 * wd, wd / 2.0, ht / 2.0),
                            WalkerSpec(n_frames=32, seed=10 + k, turns=True, accel=1.5))
        slot = eng.add_stream(wd, ht, window=win, smooth_len=7, mode="heading")
        D = torch.from_numpy(np.stack([sw.render(j) for j in range(32)])).to(dev)
        M = torch.zeros((32, ht, wd), device=dev)
        G = torch.zeros_like(M)
        streams.append((sw, slot, D, M, G))
    for lo in range(0, 32, 16):
        for sw, slot, D, M, G in streams:
            eng.submit(slot, sw.poses[lo:lo + 16], D[lo:lo + 16], sw.K(), M[lo:lo + 16], G[lo:lo + 16])
        t = eng.tick()
    eng.wait(t)
    for k, (sw, slot, D, M, G) in enumerate(streams):
        out[f"eng{k}_M"] = M.cpu().numpy()
        out[f"eng{k}_G"] = G.cpu().numpy()
    eng.close()
    w = small_stream(seed=5, n_frames=60, window=8, smooth_len=15)
    desc = mf.mf_stream_desc_init(width=320, height=240, window=8, smooth_len=15,
                                  mode=mf.MF_MODE_HEADING, cuda_stream=1)
    M = torch.empty((40, 240, 320), device=dev)
    G = torch.empty_like(M)
    mf.mf_render_noalloc(desc, 60, torch.from_numpy(w.poses).to(dev), 40,
                         torch.from_numpy(w.depth_stack(20, 60)).to(dev), w.K(), M, G, None)
    torch.cuda.synchronize()
    out["noalloc_M"] = M.cpu().numpy()
    out["noalloc_G"] = G.cpu().numpy()
    np.savez(out_path, lib=os.path.basename(mf._mf.LIB_PATH), **out)


if __name__ == "__main__":
    main(sys.argv[1])
