"""A small, fixed GPU case for profilers: the 640x480, D = 64 scene matched
`--calls` times (64 disparities per pass, both views, consistency check,
`--vote` Eq. 4 rounds).  Usage:

    python -m paper_2203_02300_gb300.profile_case [--calls 3] [--vote 0]

Each call launches k_pack, k_prep, k_hagg, k_vagg, k_lr, then per Eq. 4
round k_hvote and k_vagg in vote mode.  Prints one line and exits 0.
"""
import argparse


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--calls", type=int, default=3)
    ap.add_argument("--vote", type=int, default=0)
    args = ap.parse_args()
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


if __name__ == "__main__":
    main()
