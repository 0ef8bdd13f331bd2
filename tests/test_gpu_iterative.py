"""Iterative unbinding (rs_config.unbind_passes) on the GPU against the oracle's passes: flags,
bound counts, halo decisions and properties bit for bit, each member's potential from its last
evaluated pass within 1e-5 relative, in the plain form, the batched form, and the batched form
with the certified tree bound forced onto small nodes (its cells rebuilt without the removed
members each pass)."""
import numpy as np
import pytest

import oracle
from helpers import gpu_ctx, small_snapshot, to_dev
from paper_2412_18629_gb300 import G_NEWTON

pytestmark = pytest.mark.gpu

PASSES = 6


def _run(s, mode, want_potential, **kw):
    import paper_2412_18629_gb300 as rs
    ctx = gpu_ctx(s, mode=mode, unbind_passes=PASSES, **kw)
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    phi, bound, _ = rs.rs_unbind(ctx, pos, vel, want_potential=want_potential)
    out = dict(labels=lab.cpu().numpy(), bound=bound.cpu().numpy(),
               phi=None if phi is None else phi.cpu().numpy(),
               props=rs.props_to_float64(rs.rs_halo_props(ctx)).cpu().numpy(),
               passes=rs.rs_unbind_passes(ctx), tree=rs.rs_tree_stats(ctx))
    ctx.close()
    return out


@pytest.mark.parametrize("mode,want_potential,kw", [
    ("plain", True, {}), ("batched", True, {}), ("batched", False, {"tree_min": 128})])
def test_iterative_unbinding_matches_the_oracle(mode, want_potential, kw):
    s = small_snapshot(1 << 15, 32.0, 101, n_max=5000)
    g = _run(s, mode, want_potential, **kw)
    h = oracle.hierarchy(s["pos"], s["vel"], s["ids"], g["labels"], s["box"])
    ub = oracle.unbind(h["member_off"], h["member_idx"], s["pos"], s["vel"], s["box"],
                       s["softening"], G_NEWTON, s["particle_mass"], passes=PASSES)
    one = oracle.unbind(h["member_off"], h["member_idx"], s["pos"], s["vel"], s["box"],
                        s["softening"], G_NEWTON, s["particle_mass"], want_phi=False)
    assert (one["bound"] != ub["bound"]).sum() > 0      # the passes change flags here
    assert g["passes"] >= 2
    assert np.array_equal(g["bound"], ub["bound"])
    P = g["props"]
    assert np.array_equal(P[:, 1], ub["n_bound"].astype(np.float64))
    assert np.array_equal(P[:, 2], ub["is_halo"].astype(np.float64))
    po = oracle.props(h["member_off"], h["member_idx"], s["pos"], s["vel"], ub["bound"],
                      ub["is_halo"], s["box"], s["particle_mass"], len(s["ids"]))
    exact = [c for c in range(20) if c != 12]
    assert np.array_equal(P[:, exact], po[:, exact])
    if want_potential:
        rel = np.abs(g["phi"].astype(np.float64) - ub["phi"]) / np.abs(ub["phi"])
        assert rel.max() <= 1e-5
    else:
        assert g["tree"]["tree_nodes"] > 0
