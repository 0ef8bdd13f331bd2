"""Parity at the two largest workloads, in the launch configuration bench.py times (batched
form, no potential output, so the certified tree bound decides the flags of nodes of 16384
members and more):

* nfw-2^25-L320-sub (2^25 particles, halos up to 5e5 members);
* nfw-2^27-L512-sub3 (2^27 particles, halos up to 2e6 members, three levels of subhalos).

The oracle cannot redo a whole snapshot of this size, so the checks are:
* FoF labels: every oracle group lying inside a sub-volume window (no member within a linking
  length of the window's faces, so its link closure is inside the window) must be exactly one
  GPU group, with the same label; over the whole snapshot every label is the smallest id of its
  group's members (the particle with that id carries it, no member has a smaller id);
* hierarchy: the whole subtree under sampled level-0 nodes, the three largest included with no
  size cap, rebuilt by the oracle from the node's own particles: node table, split parameters
  (inv_sx2, inv_sv2, l2), member lists and deepest nodes, bit for bit;
* unbinding: for every node of those subtrees with at most 20000 members the oracle's flags,
  bound counts, halo decisions and properties; for larger nodes the oracle's flags of a seeded
  random sample of members (the oracle's potential of a member is O(g))."""
import numpy as np
import pytest

import oracle
from helpers import gpu_ctx, to_dev
from paper_2412_18629_gb300 import G_NEWTON, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FULL_MAX = 20000      # nodes up to this size get the oracle's full unbinding and properties
SAMPLE_PER_NODE = 1500


@pytest.fixture(scope="module", params=["nfw-2^25-L320-sub", "nfw-2^27-L512-sub3"])
def run(request):
    import torch
    import paper_2412_18629_gb300 as rs
    s = synth.generate(synth.WORKLOADS[request.param])
    ctx = gpu_ctx(s, mode="batched")
    pos, vel, ids = to_dev(s)
    lab, _ = rs.rs_fof3d(ctx, pos, ids)
    rs.rs_fof6d(ctx, pos, vel, ids, lab)
    _, bound, _ = rs.rs_unbind(ctx, pos, vel, want_potential=False)
    props = rs.props_to_float64(rs.rs_halo_props(ctx)).cpu().numpy()
    out = dict(name=request.param, snap=s, labels=lab.cpu().numpy(),
               hier={k: v.cpu().numpy() for k, v in rs.rs_fof6d_copy(ctx).items()},
               params=rs.rs_fof6d_node_params(ctx).cpu().numpy(), bound=bound.cpu().numpy(),
               props=props, tree=rs.rs_tree_stats(ctx))
    ctx.close()
    del pos, vel, ids, lab, bound
    torch.cuda.empty_cache()
    return out


def test_labels_are_group_minima(run):
    s, lab = run["snap"], run["labels"]
    ids = s["ids"]
    assert np.all(lab <= ids)
    where = np.empty(len(ids), np.int64)
    where[ids] = np.arange(len(ids))            # ids are a permutation of 0..n-1
    assert np.array_equal(lab[where[lab]], lab)  # the particle with id = label carries it


def test_labels_in_window_match_the_oracle(run):
    s, lab = run["snap"], run["labels"]
    L = float(s["box"])
    w = L / 4.0
    ll = float(s["link_length"])
    inside = np.all(s["pos"] < np.float32(w), axis=1)
    sub = np.flatnonzero(inside)
    lab_o = oracle.fof3d_grid(s["pos"][sub], s["ids"][sub], s["box"], s["link_length"])
    # complete groups: no member within a linking length of the window's faces
    p = s["pos"][sub].astype(np.float64)
    edge = np.any((p < 1.001 * ll) | (p >= w - 1.001 * ll), axis=1)
    u, inv = np.unique(lab_o, return_inverse=True)
    touched = np.zeros(len(u), bool)
    touched[inv[edge]] = True
    ok = ~touched[inv]
    assert ok.sum() > 0.5 * len(sub)
    assert np.array_equal(lab[sub][ok], lab_o[ok])
    # and each complete group is the whole GPU group of that label (no member outside it)
    labs, cnt_o = np.unique(lab_o[ok], return_counts=True)
    gl, gcnt = np.unique(lab, return_counts=True)
    idx = np.searchsorted(gl, labs)
    assert np.array_equal(gl[idx], labs) and np.array_equal(gcnt[idx], cnt_o)


def _children(parent):
    kids = {}
    for c, pq in enumerate(parent):
        if pq >= 0:
            kids.setdefault(int(pq), []).append(c)
    return kids


def _subtree(kids, q):
    out, frontier = [q], [q]
    while frontier:
        nxt = [c for f in frontier for c in kids.get(f, [])]
        out += nxt
        frontier = nxt
    return sorted(out)


def _sampled_roots(h, rng):
    size, level = h["size"], h["level"]
    roots = np.flatnonzero(level == 0)
    big = roots[np.argsort(-size[roots], kind="stable")[:3]]
    mid = roots[(size[roots] >= 1000) & (size[roots] <= 100000)]
    has_kids = np.zeros(len(size), bool)
    has_kids[h["parent"][h["parent"] >= 0]] = True
    nested = roots[has_kids[roots] & (size[roots] <= 100000)]
    pick = np.r_[big, rng.choice(mid, min(3, len(mid)), replace=False),
                 rng.choice(nested, min(3, len(nested)), replace=False)]
    return np.unique(pick)


@pytest.fixture(scope="module")
def subtrees(run):
    """Per sampled root: (GPU subtree node indices, oracle hierarchy of the root's particles,
    the root's particles)."""
    h = run["hier"]
    s = run["snap"]
    rng = np.random.default_rng(27)
    kids = _children(h["parent"])
    out = []
    for q in _sampled_roots(h, rng):
        mem = h["member_idx"][h["member_off"][q]:h["member_off"][q + 1]]
        lab = np.full(len(mem), s["ids"][mem].min(), np.int64)
        ho = oracle.hierarchy(s["pos"][mem], s["vel"][mem], s["ids"][mem], lab, s["box"])
        out.append((int(q), _subtree(kids, int(q)), ho, mem))
    return out


def test_sampled_subtrees_match_the_oracle(run, subtrees):
    h, prm = run["hier"], run["params"]
    largest = max(h["size"][h["level"] == 0])
    assert any(h["size"][q] == largest for q, _, _, _ in subtrees)
    for q, nodes, ho, mem in subtrees:
        nodes = np.asarray(nodes)
        loc = {int(g): i for i, g in enumerate(nodes)}
        assert len(nodes) == len(ho["size"]), q
        assert np.array_equal(h["size"][nodes], ho["size"]), q
        assert np.array_equal(h["level"][nodes] - h["level"][q], ho["level"]), q
        assert np.array_equal(h["min_id"][nodes], ho["min_id"]), q
        par = np.array([loc.get(int(p), -1) if i else -1 for i, p in enumerate(h["parent"][nodes])])
        assert np.array_equal(par, ho["parent"]), q
        assert np.array_equal(prm[nodes, :3], ho["params"]), q
        for i, g in enumerate(nodes):
            gm = h["member_idx"][h["member_off"][g]:h["member_off"][g + 1]]
            om = mem[ho["member_idx"][ho["member_off"][i]:ho["member_off"][i + 1]]]
            assert np.array_equal(gm, om), (q, g)
        deep_o = np.where(ho["deepest"] >= 0, nodes[np.maximum(ho["deepest"], 0)], -1)
        assert np.array_equal(h["deepest"][mem], deep_o), q


def test_sampled_flags_match_the_oracle(run, subtrees):
    h, s = run["hier"], run["snap"]
    rng = np.random.default_rng(28)
    off, midx = h["member_off"], h["member_idx"]
    full = [g for _, nodes, _, _ in subtrees for g in nodes if h["size"][g] <= FULL_MAX]
    big = [g for _, nodes, _, _ in subtrees for g in nodes if h["size"][g] > FULL_MAX]
    assert big, "no node above the full-check size"
    # complete unbinding and properties of the smaller nodes
    full = np.asarray(sorted(set(full)))
    sizes = h["size"][full]
    coff = np.r_[0, np.cumsum(sizes)]
    cmem = np.concatenate([midx[off[g]:off[g + 1]] for g in full])
    ub = oracle.unbind(coff, cmem, s["pos"], s["vel"], s["box"], s["softening"], G_NEWTON,
                       s["particle_mass"], want_phi=False)
    gb = np.concatenate([run["bound"][off[g]:off[g + 1]] for g in full])
    assert np.array_equal(gb, ub["bound"])
    po = oracle.props(coff, cmem, s["pos"], s["vel"], ub["bound"], ub["is_halo"], s["box"],
                      s["particle_mass"], len(s["ids"]))
    P = run["props"][full]
    exact = [c for c in range(20) if c != 12]
    assert np.array_equal(P[:, exact], po[:, exact])
    np.testing.assert_allclose(P[:, 12], po[:, 12], rtol=4 * 2.0 ** -52, atol=0)
    # sampled members of the larger nodes
    for g in sorted(set(big)):
        mem = midx[off[g]:off[g + 1]]
        pick = np.sort(rng.choice(len(mem), min(SAMPLE_PER_NODE, len(mem)), replace=False))
        _, bo = oracle.unbind_sample(mem, s["pos"], s["vel"], s["box"], s["softening"], G_NEWTON,
                                     s["particle_mass"], pick)
        assert np.array_equal(run["bound"][off[g]:off[g + 1]][pick], bo), g
        P = run["props"][g]
        assert P[1] == run["bound"][off[g]:off[g + 1]].sum()


def test_tree_bound_decided_most_members(run):
    t = run["tree"]
    assert t["tree_nodes"] > 0 and t["decided_by_bound"] >= 0.8 * t["tree_members"], t
