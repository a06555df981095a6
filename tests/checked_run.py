"""One fixed GPU workload whose results the checked-build test compares
between the library and its range-checked variant (the variant is chosen by
the CWTHF_CHECKED environment variable when the binding loads the library, so
the checked run happens in a child process).  Run as a script it prints the
results as one JSON line."""
import json
import sys


def run() -> dict:
    import numpy as np
    import torch

    import paper_2501_10622_gb300 as pkg
    from paper_2501_10622_gb300 import synth
    dev = torch.device("cuda", 0)
    out = {}
    ctx = pkg.Context(0, max_ng=96, max_np=1 << 18, max_scales=3, unbind=True)
    try:
        out["checked"] = ctx.debug_get(pkg._lib.DEBUG_CHECKED)
        # find over three scales on a clumped box
        L = 50.0
        pos = synth.clumped_box(1 << 17, L, 60, seed=21, device=dev)
        hid, cat, nh = ctx.find(pos, L, 64, [pkg.default_params(w) for w in (2.0, 3.0, 4.0)])
        out["find_status"] = ctx.sync()
        out["find_n_halo"] = nh.cpu().tolist()
        out["find_ids"] = int((hid.to(torch.int64) * 31 + 7).remainder(1000003).sum().item())
        # a dense core: tiles split into parts
        core = torch.rand((60000, 3), generator=torch.Generator().manual_seed(3)) * 0.3 + 8.0
        dense = torch.cat([core, synth.clumped_box(20000, L, 5, seed=4)]).to(dev)
        g = ctx.deposit(dense, L, 96)
        out["deposit_status"] = ctx.sync()
        out["deposit"] = int((g % 1000003).sum().item())
        # the multi-scale loop with the self-boundness check, most groups on the whole-grid path
        pos2, vel2 = synth.clumped_box(24000, 40.0, 40, seed=2, velocities=True)
        ctx.debug_set(pkg._lib.DEBUG_UNBIND_GRID_MIN, 40)
        hid2, cat2, nh2 = ctx.find_multiscale(pos2.to(dev), 40.0, [1.5, 2.5, 3.5], [24, 36, 48],
                                              mass_unit=synth.particle_mass(24000, 40.0), vel=vel2.to(dev))
        out["ms_status"] = ctx.sync()
        out["ms_n_halo"] = int(nh2[0])
        out["ms_ids"] = [int(x) for x in np.bincount(hid2.cpu().numpy() + 1)[:64]]
    finally:
        ctx.close()
    return out


if __name__ == "__main__":
    sys.stdout.write(json.dumps(run()) + "\n")
