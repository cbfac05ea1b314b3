"""The identities the team form of the batched kernels rests on, checked in
FP64 on random trees (host-side mathematics; no kernel and no oracle code).

For world poses R_i = R_p R_local,i and P_i = P_p + R_p P_local,i, the pose
cotangents passed through every joint transform leaves first,
    R_bar_p += R_bar_c R_local,c^T + P_bar_c P_local,c^T,   P_bar_p += P_bar_c,
equal the subtree sums of the world-frame moments Q_k = R_bar_k R_k^T +
P_bar_k P_k^T of each link's own cotangents:
    R_bar_p = (sum_sub Q - (sum_sub P_bar) P_p^T) R_p.
The root-first recursions V_i = V_p + u_i and A_i = A_p + c_i are ancestor
sums, and the leaves-first totals are subtree sums, both in link order when
parents come first."""
import numpy as np
import pytest


def random_tree(rng, L):
    parent = np.array([-1] + [int(rng.integers(0, i)) for i in range(1, L)])
    if L > 3:   # a second root, as the model rules allow
        parent[3] = -1
    return parent


def random_rotation(rng):
    q = rng.normal(size=4)
    x, y, z, w = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def world_poses(parent, Rl, Pl):
    R, P = Rl.copy(), Pl.copy()
    for i in range(len(parent)):
        p = parent[i]
        if p >= 0:
            R[i] = R[p] @ Rl[i]
            P[i] = P[p] + R[p] @ Pl[i]
    return R, P


@pytest.mark.parametrize("seed,L", [(0, 2), (1, 9), (2, 13), (3, 22), (4, 32)])
def test_pose_cotangents_telescope_into_world_frame_sums(seed, L):
    rng = np.random.default_rng(seed)
    parent = random_tree(rng, L)
    Rl = np.stack([random_rotation(rng) for _ in range(L)])
    Pl = rng.normal(scale=0.3, size=(L, 3))
    R, P = world_poses(parent, Rl, Pl)
    Rb_own = rng.normal(size=(L, 3, 3))
    Pb_own = rng.normal(size=(L, 3))
    # through the joint transforms, children before parents
    Rb, Pb = Rb_own.copy(), Pb_own.copy()
    for c in range(L - 1, -1, -1):
        p = parent[c]
        if p >= 0:
            Rb[p] += Rb[c] @ Rl[c].T + np.outer(Pb[c], Pl[c])
            Pb[p] += Pb[c]
    # subtree sums of the world-frame moments
    Q = np.einsum("kab,kcb->kac", Rb_own, R) + np.einsum("ka,kb->kab", Pb_own, P)
    SQ, SP = Q.copy(), Pb_own.copy()
    for i in range(L - 1, 0, -1):
        if parent[i] >= 0:
            SQ[parent[i]] += SQ[i]
            SP[parent[i]] += SP[i]
    Rb_world = np.einsum("kab,kbc->kac", SQ - np.einsum("ka,kb->kab", SP, P), R)
    np.testing.assert_allclose(Rb_world, Rb, rtol=0, atol=1e-11 * (1 + np.abs(Rb).max()))
    np.testing.assert_allclose(SP, Pb, rtol=0, atol=1e-12 * (1 + np.abs(Pb).max()))


@pytest.mark.parametrize("seed,L", [(5, 9), (6, 22)])
def test_recursions_are_ancestor_and_subtree_sums(seed, L):
    rng = np.random.default_rng(seed)
    parent = random_tree(rng, L)
    own = rng.normal(size=(L, 6))
    # root first: x_i = x_p + own_i (a root starts from its own term)
    rec = np.zeros_like(own)
    for i in range(L):
        rec[i] = own[i] + (rec[parent[i]] if parent[i] >= 0 else 0.0)
    anc = own.copy()
    for i in range(1, L):
        if parent[i] >= 0:
            anc[i] += anc[parent[i]]
    np.testing.assert_allclose(anc, rec, rtol=0, atol=1e-12)
    # leaves first: totals over each subtree, by explicit descendant sets
    desc = [{i} for i in range(L)]
    for i in range(L - 1, 0, -1):
        if parent[i] >= 0:
            desc[parent[i]] |= desc[i]
    tot = np.stack([own[sorted(d)].sum(0) for d in desc])
    sub = own.copy()
    for i in range(L - 1, 0, -1):
        if parent[i] >= 0:
            sub[parent[i]] += sub[i]
    np.testing.assert_allclose(sub, tot, rtol=0, atol=1e-12)


def test_pose_rows_need_only_the_parents_row():
    """Row r of R_p R_local and P_p[r] + (row r of R_p) . P_local use row r of
    the parent's pose only (the poses by rows)."""
    rng = np.random.default_rng(7)
    parent = random_tree(rng, 12)
    Rl = np.stack([random_rotation(rng) for _ in range(12)])
    Pl = rng.normal(size=(12, 3))
    R, P = world_poses(parent, Rl, Pl)
    for r in range(3):
        row, pr = Rl[:, r, :].copy(), Pl[:, r].copy()
        for i in range(12):
            p = parent[i]
            if p >= 0:
                row[i] = row[p] @ Rl[i]
                pr[i] = pr[p] + row[p] @ Pl[i]
        np.testing.assert_allclose(row, R[:, r, :], rtol=0, atol=1e-12)
        np.testing.assert_allclose(pr, P[:, r], rtol=0, atol=1e-12)
