"""A small, fixed GPU case for profilers: the 640x480, D = 64 scene matched
`--calls` times (64 disparities per pass, both views, consistency check,
`--vote` Eq. 4 rounds).  Usage:

    python -m paper_2203_02300_gb300.profile_case [--calls 3] [--vote 0] [--densify]

Each call launches k_pack, k_prep, k_hagg, k_vagg, k_lr, then per Eq. 4
round k_hvote and k_vagg in vote mode.  With --densify the case is instead a
1280x720 frame: its sparse depth (dco_stereo_depth, 640x360 D = 64) densified
(Sect. 6) `--calls` times with per-kernel profiling on (plain launches).
Prints one line and exits 0.
"""
import argparse


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--calls", type=int, default=3)
    ap.add_argument("--vote", type=int, default=0)
    ap.add_argument("--densify", action="store_true")
    args = ap.parse_args()
    if args.densify:
        return densify_case(args.calls)
    import torch
    from . import binding, build, scenes
    build.build()
    s = scenes.config_scene(2)
    L = torch.from_numpy(s.left).cuda()
    R = torch.from_numpy(s.right).cuda()
    out = torch.empty((s.H, s.W), dtype=torch.int16, device="cuda")
    p = binding.Params.default(d_chunk=64, vote_iters=args.vote)
    with binding.Stereo(0) as st:
        for _ in range(args.calls):
            st.match(L, R, s.D, p, out)
        torch.cuda.synchronize()
        st.sync_status()
    print(f"profile_case ok: {args.calls} calls, {args.vote} Eq. 4 rounds, max disparity {int(out.max())}")


def densify_case(calls: int) -> None:
    import numpy as np
    import torch
    from . import binding, build, scenes
    build.build()
    s = scenes.plane_scene(1280, 720, 128, 12, seed=scenes.seed_for(2, 950), drange=(4, 120), slanted=True,
                           noise_sigma=2.0)
    g = s.disp
    B = ((np.abs(np.diff(g, axis=1, append=g[:, -1:])) > 1) | (np.abs(np.diff(g, axis=0, append=g[-1:])) > 1))
    Y = s.left.astype(np.float32).mean(axis=2)
    gm = np.hypot(*np.gradient(Y))
    with binding.Stereo(0) as st:
        z = st.depth(torch.from_numpy(s.left).cuda(), torch.from_numpy(s.right).cuda(), 64, 700.0, 0.12)
        Bd = torch.from_numpy(B.astype(np.uint8)).cuda()
        mi = torch.from_numpy((gm / gm.max()).astype(np.float32)).cuda()
        st.set_profiling(True)
        for _ in range(calls):
            out = st.densify(z, Bd, torch.ones_like(mi), mi)
        torch.cuda.synchronize()
        it, rel = st.densify_stats()
    print(f"profile_case ok: densify 1280x720, {calls} solves, {it} iterations, relative residual {rel:.2e}, "
          f"mean depth {float(out.mean()):.3f}")


if __name__ == "__main__":
    main()
