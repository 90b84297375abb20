"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these retypes the oracle's formulas: each checks a closed form, an
invariant, a special case that reduces to a textbook routine, a hand-computed
value or a brute-force count, chosen so that a dropped term, a wrong sign, a
swapped index or a transposed operand in the oracle fails at least one.
"""

import numpy as np
import pytest
from scipy import stats

pytestmark = []

CFG1 = dict(L=8, F=2, log2T=14, n_min=16, n_max=256, width=32, hidden=2, lambda_d=0.1, lambda_sigma=0.0)
CFG2 = dict(L=16, F=2, log2T=19, n_min=16, n_max=2048, width=64, hidden=2, lambda_d=0.1, lambda_sigma=0.0)


# ----------------------------------------------------------------- hash grid
def test_level_resolutions_hand_computed(orc):
    # b = 16^(1/7) = 1.48599...; 16 b^l = 16, 23.78, 35.33, 52.50, 78.02, 115.93, 172.27, 256
    a = orc.Arch(**CFG1)
    assert [orc.level_res(a, l) for l in range(8)] == [16, 23, 35, 52, 78, 115, 172, 256]
    # b = 128^(1/15) = 1.38191...; the finest level must land exactly on N_max
    a2 = orc.Arch(**CFG2)
    res = [orc.level_res(a2, l) for l in range(16)]
    assert res[0] == 16 and res[-1] == 2048
    assert res == [16, 22, 30, 42, 58, 80, 111, 153, 212, 294, 406, 561, 776, 1072, 1482, 2048]


def test_dense_hashed_split_and_sizes(orc):
    # cfg 1: (17^3 = 4913) and (24^3 = 13824) fit in 2^14 = 16384; 36^3 = 46656 does not
    a = orc.Arch(**CFG1)
    assert [orc.level_dense(a, l) for l in range(8)] == [True, True] + [False] * 6
    assert [orc.level_entries(a, l) for l in range(2)] == [4913, 13824]
    # storage pads every level to a multiple of 8 entries: 4913 -> 4920
    assert orc.n_hash_params(a) == 2 * (4920 + 13824 + 6 * 16384)
    assert [orc.level_offset(a, l) for l in range(3)] == [0, 2 * 4920, 2 * (4920 + 13824)]
    # cfg 2: 17^3, 23^3, 31^3, 43^3, 59^3 fit in 2^19; 81^3 = 531441 > 524288
    a2 = orc.Arch(**CFG2)
    assert [orc.level_dense(a2, l) for l in range(16)] == [True] * 5 + [False] * 11
    assert [orc.level_entries(a2, l) for l in range(5)] == [4913, 12167, 29791, 79507, 205379]
    assert orc.n_hash_params(a2) == 2 * (4920 + 12168 + 29792 + 79512 + 205384 + 11 * 524288)
    assert all(orc.level_offset(a2, l) % 16 == 0 for l in range(17))  # 8 entries x 2 features
    # MLP: 32->64, 64->64, 64->4 without biases
    assert orc.n_mlp_params(a2) == 32 * 64 + 64 * 64 + 4 * 64
    assert orc.param_count(a2) == orc.n_hash_params(a2) + 6400


def test_hash_index_hand_values(orc):
    a = orc.Arch(**CFG1)
    l = 5  # hashed level, T = 2^14
    assert orc.grid_index(a, l, 1, 0, 0) == 1  # pi_1 = 1
    assert orc.grid_index(a, l, 0, 1, 0) == 0x9E3779B1 & 0x3FFF  # 2654435761 mod 2^14 = 14769
    assert orc.grid_index(a, l, 0, 0, 1) == 0x30025795 & 0x3FFF  # 805459861 mod 2^14 = 6037
    assert orc.grid_index(a, l, 1, 1, 1) == (1 ^ 0x39B1 ^ 0x1795)  # = 11813
    # wraparound of the uint32 products
    assert orc.grid_index(a, l, 0, 3, 0) == (3 * 2654435761 % 2**32) & 0x3FFF


def test_dense_index_is_a_bijection(orc):
    a = orc.Arch(**CFG1)
    for l in (0, 1):
        n1 = orc.level_res(a, l) + 1
        seen = np.zeros(n1 ** 3, dtype=np.int32)
        for z in range(n1):
            for y in range(n1):
                for x in (0, 1, n1 - 1):
                    seen[orc.grid_index(a, l, x, y, z)] += 1
        # x covers 0,1,N per (y,z): 3 n1^2 distinct entries, never out of range
        assert seen.sum() == 3 * n1 * n1 and seen.max() == 1
        assert orc.grid_index(a, l, n1 - 1, n1 - 1, n1 - 1) == n1 ** 3 - 1


def test_hashed_index_x_is_a_permutation(orc):
    # with pi_1 = 1, x -> x xor h(y, z) mod T is a bijection of [0, T) for fixed (y, z)
    a = orc.Arch(L=2, F=2, log2T=8, n_min=16, n_max=600, width=16, hidden=1)
    assert not orc.level_dense(a, 1)
    idx = {orc.grid_index(a, 1, x, 7, 11) for x in range(256)}
    assert idx == set(range(256))


# -------------------------------------------------------------------- encoding
def _dense_arch(orc):
    # every level collision-free: (8+1)^3 = 729 <= 4096
    a = orc.Arch(L=3, F=2, log2T=12, n_min=2, n_max=8, width=16, hidden=1)
    assert all(orc.level_dense(a, l) for l in range(3))
    return a


def test_encoding_reproduces_affine_fields(orc):
    a = _dense_arch(orc)
    rng = np.random.default_rng(0)
    theta = np.zeros(orc.param_count(a))
    coef = rng.normal(size=(a.L, a.F, 4))  # feature f of level l = c0 + c . vertex / N_l
    for l in range(a.L):
        n = orc.level_res(a, l)
        off = orc.level_offset(a, l)
        for z in range(n + 1):
            for y in range(n + 1):
                for x in range(n + 1):
                    i = orc.grid_index(a, l, x, y, z)
                    for f in range(a.F):
                        c = coef[l, f]
                        theta[off + i * a.F + f] = c[0] + c[1] * x / n + c[2] * y / n + c[3] * z / n
    for p in rng.random((50, 3)):
        enc = orc.encode(a, theta, p)
        want = [coef[l, f, 0] + coef[l, f, 1:] @ p for l in range(a.L) for f in range(a.F)]
        np.testing.assert_allclose(enc, want, rtol=0, atol=1e-12)
    # p on the far faces uses the last cell with weight 1 (corner clamp)
    enc = orc.encode(a, theta, np.ones(3))
    want = [coef[l, f, 0] + coef[l, f, 1:].sum() for l in range(a.L) for f in range(a.F)]
    np.testing.assert_allclose(enc, want, atol=1e-12)


def test_encoding_partition_of_unity_and_vertex_lookup(orc):
    a = orc.Arch(**CFG1)
    rng = np.random.default_rng(1)
    theta = np.zeros(orc.param_count(a))
    # constant tables -> every level's encoding equals the constant (weights sum to 1)
    for l in range(a.L):
        off = orc.level_offset(a, l)
        n = orc.level_entries(a, l)
        theta[off:off + n * a.F].reshape(n, a.F)[:] = [l + 1.0, -(l + 1.0)]
    for p in rng.random((20, 3)):
        enc = orc.encode(a, theta, p).reshape(a.L, a.F)
        np.testing.assert_allclose(enc[:, 0], np.arange(1, a.L + 1), atol=1e-12)
        np.testing.assert_allclose(enc[:, 1], -np.arange(1, a.L + 1), atol=1e-12)
    # a table holding its own index, probed exactly on a vertex, returns the hash of that vertex
    l = 5
    n = orc.level_res(a, l)
    off = orc.level_offset(a, l)
    theta[off:off + orc.level_entries(a, l) * a.F] = np.repeat(np.arange(orc.level_entries(a, l)), a.F)
    v = (3, 5, 7)
    p = np.array(v, dtype=np.float64) / n
    enc = orc.encode(a, theta, p).reshape(a.L, a.F)
    assert enc[l, 0] == float((3 ^ (5 * 2654435761) ^ (7 * 805459861)) % 2**32 & 0x3FFF)


def test_encoding_backward_is_the_transpose(orc):
    # <J x, y> = <x, J^T y> for the linear map theta -> enc
    a = orc.Arch(L=4, F=2, log2T=12, n_min=4, n_max=64, width=16, hidden=1)
    rng = np.random.default_rng(2)
    n = orc.param_count(a)
    for p in rng.random((5, 3)):
        x = rng.normal(size=n)
        y = rng.normal(size=a.n_in)
        lhs = orc.encode(a, x, p) @ y
        rhs = orc.encode_backward(a, p, y, n) @ x
        assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1)


# ------------------------------------------------------------------------- MLP
def test_mlp_matches_numpy_matmul_chain(orc):
    a = orc.Arch(**CFG2)
    rng = np.random.default_rng(3)
    theta = rng.normal(size=orc.param_count(a)) * 0.3
    Ws = []
    for layer, (o_, i_) in enumerate(a.mlp_shapes()):
        off = orc.mlp_offset(a, layer)
        Ws.append(theta[off:off + o_ * i_].reshape(o_, i_))
    for _ in range(5):
        x = rng.normal(size=a.n_in)
        h = x
        hs = []
        for W in Ws[:-1]:
            h = np.maximum(W @ h, 0.0)
            hs.append(h)
        out = Ws[-1] @ h
        acts, o = orc.mlp_forward(a, theta, x)
        np.testing.assert_allclose(o, out, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(acts, np.concatenate(hs), rtol=1e-12, atol=1e-12)
        # backward = transposed products with the ReLU masks
        dout = rng.normal(size=4)
        g, denc = orc.mlp_backward(a, theta, x, acts, dout)
        dh = Ws[-1].T @ dout
        gw = [np.outer(dout, hs[-1])]
        for k in range(len(Ws) - 2, -1, -1):
            dh = dh * (hs[k] > 0)
            below = hs[k - 1] if k > 0 else x
            gw.append(np.outer(dh, below))
            dh = Ws[k].T @ dh
        np.testing.assert_allclose(denc, dh, rtol=1e-10, atol=1e-12)
        for layer, gwl in zip(range(len(Ws) - 1, -1, -1), gw):
            off = orc.mlp_offset(a, layer)
            np.testing.assert_allclose(g[off:off + gwl.size], gwl.ravel(), rtol=1e-10, atol=1e-12)


def test_mlp_zero_weights(orc):
    a = orc.Arch(**CFG1)
    theta = np.zeros(orc.param_count(a))
    acts, out = orc.mlp_forward(a, theta, np.ones(a.n_in))
    assert np.all(out == 0) and np.all(acts == 0)


# -------------------------------------------------------------------- ray box
def test_ray_box_cases(orc):
    hit, tn, tf = orc.ray_box([-1.0, 0.5, 0.5], [1.0, 0.0, 0.0])
    assert hit and tn == 1.0 and tf == 2.0
    hit, tn, tf = orc.ray_box([0.5, 0.5, 0.5], [0.0, 0.0, 1.0])  # starts inside
    assert hit and tn == 0.0 and tf == 0.5
    s = 1 / np.sqrt(3)
    hit, tn, tf = orc.ray_box([-1.0, -1.0, -1.0], [s, s, s])  # diagonal
    assert hit and abs(tn - np.sqrt(3)) < 1e-12 and abs(tf - 2 * np.sqrt(3)) < 1e-12
    assert not orc.ray_box([-1.0, 2.0, 0.5], [1.0, 0.0, 0.0])[0]  # parallel, outside in y
    assert not orc.ray_box([2.0, 0.5, 0.5], [1.0, 0.0, 0.0])[0]  # points away


# --------------------------------------------------------------- prior lookup
def test_prior_lookup_affine_and_centres(orc):
    R = 8
    c = (np.arange(R) + 0.5) / R
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    grid = 1.5 + 2.0 * x - 3.0 * y + 0.5 * z
    rng = np.random.default_rng(4)
    for p in rng.uniform(0.5 / R, 1 - 0.5 / R, (50, 3)):
        assert abs(orc.prior_lookup(grid, p) - (1.5 + 2 * p[0] - 3 * p[1] + 0.5 * p[2])) < 1e-12
    g2 = rng.random((R, R, R))
    for (i, j, k) in [(0, 0, 0), (3, 5, 7), (7, 7, 7), (2, 6, 1)]:
        p = np.array([(i + 0.5) / R, (j + 0.5) / R, (k + 0.5) / R])
        assert abs(orc.prior_lookup(g2, p) - g2[k, j, i]) < 1e-12
    # outside the centre lattice the value is held constant (clamped)
    assert abs(orc.prior_lookup(g2, [0.0, 0.0, 0.0]) - g2[0, 0, 0]) < 1e-12
    assert abs(orc.prior_lookup(g2, [1.0, 1.0, 1.0]) - g2[-1, -1, -1]) < 1e-12


# ------------------------------------------------------------------- sampling
def _straight_ray():
    return np.array([-1.0, 0.5, 0.5]), np.array([1.0, 0.0, 0.0])  # tn = 1, tf = 2


def test_constant_density_slab_closed_form(orc):
    R, nc, nr = 8, 32, 16
    sigma0 = 3.0
    grid = np.full((R, R, R), sigma0)
    o, d = _straight_ray()
    u = (np.arange(nr) + 0.5) / nr
    out = orc.sample_ray(grid, o, d, nc, nr, 1e-4, u)
    delta = 1.0 / nc
    i = np.arange(nc)
    rho = (1 - np.exp(-sigma0 * delta)) * np.exp(-sigma0 * delta * i)  # T at depth s = exp(-sigma s)
    np.testing.assert_allclose(out["probe_sigma"], sigma0, rtol=1e-14)
    np.testing.assert_allclose(out["rho_term"], rho, rtol=1e-12)
    k = np.arange(nc + 1)
    cdf = (1 - np.exp(-sigma0 * delta * k)) / (1 - np.exp(-sigma0 * delta * nc))
    np.testing.assert_allclose(out["cdf"], cdf, rtol=1e-12, atol=1e-15)
    assert not out["escape"] and out["tn"] == 1.0 and out["tf"] == 2.0
    # inverse of the piecewise-linear CDF evaluated at the samples gives back u
    t = out["t"]
    s = (t - 1.0) / delta
    cdf_at = np.interp(s, k, cdf)
    np.testing.assert_allclose(cdf_at, u, atol=1e-12)


def test_cdf_invert_dyadic_edges_and_empty_bins(orc):
    # masses in multiples of 2^-10 so every edge is exact
    mass = np.array([0, 256, 0, 128, 512, 0, 0, 128], dtype=np.float64) / 1024
    cdf = np.concatenate([[0.0], np.cumsum(mass)])
    u = np.array([0.0, 0.25 - 2**-20, 0.25, 0.375, 0.5, 0.875, 0.875 + 2**-11, 1 - 2**-24])
    bins, t = orc.cdf_invert(cdf, u, 2.0, 10.0)
    # u = 0 -> first non-empty bin; u on an edge -> the next non-empty bin (strict >)
    assert bins.tolist() == [1, 1, 3, 4, 4, 7, 7, 7]
    assert 0 not in bins and 2 not in bins and 5 not in bins and 6 not in bins
    # positions: bin b covers [2 + b, 3 + b]; linear inside the bin
    assert t[0] == 3.0 and t[2] == 5.0 and t[3] == 6.0
    assert abs(t[4] - (6.0 + 0.25)) < 1e-15  # (0.5 - 0.375) / 0.5 = 1/4 of bin 4


def test_escape_gives_uniform_bins(orc):
    R, nc, nr = 8, 32, 32
    grid = np.zeros((R, R, R))
    o, d = _straight_ray()
    u = np.random.default_rng(5).random(nr)
    out = orc.sample_ray(grid, o, d, nc, nr, 1e-4, u)
    assert out["escape"]
    np.testing.assert_array_equal(out["bins"], np.floor(u * nc).astype(int))
    np.testing.assert_allclose(out["t"], 1.0 + u, atol=1e-14)
    # a density just under / over the threshold: total = 1 - exp(-sigma * 1)
    for sig, esc in [(0.99e-4, True), (1.01e-4, False)]:
        out = orc.sample_ray(np.full((R, R, R), sig), o, d, nc, nr, 1e-4, u)
        assert out["escape"] == esc


def test_one_hot_with_opaque_voxels(orc):
    R, nc, nr = 16, 32, 16
    grid = np.zeros((R, R, R))
    grid[:, :, 10:] = 1e30  # x >= 10/16 opaque
    o, d = _straight_ray()
    u = np.random.default_rng(6).random(nr)
    out = orc.sample_ray(grid, o, d, nc, nr, 1e-4, u)
    b = out["bins"]
    assert np.all(b == b[0])
    assert out["probe_sigma"][b[0]] > 0 and np.all(out["probe_sigma"][:b[0]] == 0)
    assert out["rho_term"][b[0]] == 1.0 and np.all(np.delete(out["rho_term"], b[0]) == 0)


def test_sample_counts_match_bin_masses(orc):
    R, nc = 8, 16
    rng = np.random.default_rng(7)
    grid = rng.uniform(0, 6, (R, R, R))
    o, d = _straight_ray()
    nr = 64
    u = (np.arange(nr) + 0.5) / nr
    out = orc.sample_ray(grid, o, d, nc, nr, 1e-4, u)
    p = np.diff(out["cdf"])
    counts = np.bincount(out["bins"], minlength=nc)
    assert np.all(np.abs(counts - nr * p) <= 1.0 + 1e-9)
    # chi^2 of 10^6 random draws against the bin masses
    uu = rng.random(1_000_000)
    bins, _ = orc.cdf_invert(out["cdf"], uu, out["tn"], out["tf"])
    counts = np.bincount(bins, minlength=nc)
    keep = p > 0
    pval = stats.chisquare(counts[keep], 1_000_000 * p[keep]).pvalue
    assert pval > 1e-4, pval


# ------------------------------------------------------------------ rendering
def test_composite_closed_forms(orc):
    nr = 12
    t = np.linspace(1.0, 2.0, nr, endpoint=False)
    tf = 2.0
    rng = np.random.default_rng(8)
    c = rng.random((nr, 3))
    # sigma = 0 -> nothing
    w, Cc, D, A = orc.composite(np.zeros(nr), c, t, tf)
    assert A == 0 and D == 0 and np.all(Cc == 0)
    # constant density: A = 1 - exp(-sigma (tf - t_0)); w_k = exp(-sigma (t_k - t_0)) (1 - exp(-sigma delta))
    s0 = 2.5
    w, Cc, D, A = orc.composite(np.full(nr, s0), c, t, tf)
    assert abs(A - (1 - np.exp(-s0 * (tf - t[0])))) < 1e-14
    dl = np.diff(np.append(t, tf))
    np.testing.assert_allclose(w, np.exp(-s0 * (t - t[0])) * (1 - np.exp(-s0 * dl)), rtol=1e-13)
    np.testing.assert_allclose(Cc, w @ c, rtol=1e-13)
    assert abs(D - w @ t) < 1e-13
    # constant colour -> C = A c
    w, Cc, D, A = orc.composite(rng.uniform(0, 4, nr), np.tile([0.2, 0.5, 0.9], (nr, 1)), t, tf)
    np.testing.assert_allclose(Cc, A * np.array([0.2, 0.5, 0.9]), rtol=1e-13)
    # a single opaque sample takes all the weight
    sig = np.zeros(nr)
    sig[4] = 1e30
    w, Cc, D, A = orc.composite(sig, c, t, tf)
    assert w[4] == 1.0 and np.all(np.delete(w, 4) == 0) and D == t[4]


def test_ray_loss_hand_values(orc):
    L, gC, gD, gA = orc.ray_loss(True, [0.5, 0.2, 0.1], 1.0, 0.7, [0.4, 0.4, 0.1], 1.5, None, 0.1)
    assert abs(L - (0.01 + 0.04 + 0.0 + 0.1 * 0.5)) < 1e-15
    np.testing.assert_allclose(gC, [0.2, -0.4, 0.0], atol=1e-15)
    assert gD == -0.1 and gA == 0.0
    # background: C + (1 - A) C_rand - C_rand = C - A C_rand = (0.2, -0.2, -0.3)
    L, gC, gD, gA = orc.ray_loss(False, [0.3, 0.0, 0.0], 0.0, 0.5, [0, 0, 0], 0.0, [0.2, 0.4, 0.6], 0.1)
    assert abs(L - 0.17) < 1e-15
    np.testing.assert_allclose(gC, [0.4, -0.4, -0.6], atol=1e-15)
    assert gD == 0.0 and abs(gA - (-(0.4 * 0.2 - 0.4 * 0.4 - 0.6 * 0.6))) < 1e-15


def test_batch_one_ray_two_samples_by_hand(orc):
    # zero MLP -> sigma = exp(0) = 1, c = sigmoid(0) = 1/2 at every sample
    a = orc.Arch(L=2, F=2, log2T=10, n_min=2, n_max=4, width=8, hidden=1, lambda_d=0.1)
    theta = np.zeros(orc.param_count(a))
    rays = dict(o=[[-1.0, 0.5, 0.5]], d=[[1.0, 0.0, 0.0]], rgb=[[0.1, 0.2, 0.3]], depth=[1.4],
                is_obj=[1])
    t_in = np.array([[1.2, 1.7]])
    out = orc.batch(a, theta, np.zeros((2, 2, 2)), rays, 4, 2, t_in=t_in)
    w0 = 1 - np.exp(-0.5)
    w1 = np.exp(-0.5) * (1 - np.exp(-0.3))
    A = w0 + w1
    D = w0 * 1.2 + w1 * 1.7
    assert abs(out["acc"][0] - A) < 1e-15 and abs(out["depth"][0] - D) < 1e-15
    np.testing.assert_allclose(out["rgb"][0], 0.5 * A, rtol=1e-15)
    want = (0.5 * A - 0.1) ** 2 + (0.5 * A - 0.2) ** 2 + (0.5 * A - 0.3) ** 2 + 0.1 * abs(D - 1.4)
    assert abs(out["loss"] - want) < 1e-15


def _constant_field_theta(orc, a, sigma):
    """Every hash entry 1 (so every encoding feature is 1 by the partition of
    unity), W_1 = 1/IN (every hidden unit relu(1) = 1), W_out row 0 =
    ln(sigma)/W and rows 1..3 zero: density sigma and colour 1/2 everywhere."""
    nh = orc.n_hash_params(a)
    theta = np.zeros(orc.param_count(a))
    theta[:nh] = 1.0
    w1 = orc.mlp_offset(a, 0)
    theta[w1:w1 + a.width * a.n_in] = 1.0 / a.n_in
    wo = orc.mlp_offset(a, a.hidden)
    theta[wo:wo + a.width] = np.log(sigma) / a.width
    return theta


def _two_sample_weights(sigma, t0, t1, tf):
    w0 = 1 - np.exp(-sigma * (t1 - t0))
    w1 = np.exp(-sigma * (t1 - t0)) * (1 - np.exp(-sigma * (tf - t1)))
    return w0, w1


def test_batch_three_rays_with_background_and_density_penalty_by_hand(orc):
    """Eq. 8-9 over a batch of three rays, written out by hand: two object rays
    (L_c + lambda_d L_d) and one background ray (the C_rand composite and
    lambda_sigma times the sum of its samples' densities), all divided by the
    ray count R = 3.  Fails if L_sigma is charged to object rays, if its 1/R is
    dropped, or if the rays are summed instead of averaged."""
    lam_d, lam_s, sig = 0.1, 0.05, 2.0
    a = orc.Arch(L=2, F=2, log2T=10, n_min=2, n_max=4, width=8, hidden=1, lambda_d=lam_d, lambda_sigma=lam_s)
    theta = _constant_field_theta(orc, a, sig)
    # three rays along +x, y and z inside the cube: the box interval is [1, 2]
    rays = dict(o=[[-1.0, 0.5, 0.5], [-1.0, 0.3, 0.6], [-1.0, 0.7, 0.2]], d=[[1.0, 0.0, 0.0]] * 3,
                rgb=[[0.1, 0.2, 0.3], [0.6, 0.5, 0.4], [0.0, 0.0, 0.0]], depth=[1.4, 1.25, 0.0], is_obj=[1, 1, 0])
    t_in = np.array([[1.2, 1.7], [1.1, 1.5], [1.3, 1.8]])
    c_rand = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.2, 0.4, 0.6]])
    out = orc.batch(a, theta, np.zeros((2, 2, 2)), rays, 4, 2, t_in=t_in, c_rand=c_rand)
    total = 0.0
    for r in range(3):
        w0, w1 = _two_sample_weights(sig, t_in[r, 0], t_in[r, 1], 2.0)
        A = w0 + w1
        D = w0 * t_in[r, 0] + w1 * t_in[r, 1]
        C = np.full(3, 0.5 * A)
        assert abs(out["acc"][r] - A) < 1e-14 and abs(out["depth"][r] - D) < 1e-14
        np.testing.assert_allclose(out["rgb"][r], C, rtol=1e-14)
        if rays["is_obj"][r]:
            total += np.sum((C - np.array(rays["rgb"][r])) ** 2) + lam_d * abs(D - rays["depth"][r])
        else:
            # C + (1 - A) C_rand - C_rand = C - A C_rand; L_sigma = sum over the two samples of sigma
            total += np.sum((C - A * c_rand[r]) ** 2) + lam_s * (sig + sig)
    assert abs(out["loss"] - total / 3.0) < 1e-13
    # the same batch without its background ray loses exactly that ray's share
    two = {k: v[:2] for k, v in rays.items()}
    out2 = orc.batch(a, theta, np.zeros((2, 2, 2)), two, 4, 2, t_in=t_in[:2], c_rand=c_rand[:2])
    w0, w1 = _two_sample_weights(sig, 1.3, 1.8, 2.0)
    A = w0 + w1
    bg = np.sum((0.5 * A - A * c_rand[2]) ** 2) + 2 * lam_s * sig
    assert abs(3.0 * out["loss"] - 2.0 * out2["loss"] - bg) < 1e-13


# ------------------------------------------------------------------ gradients
def _fd_setup(orc, lambda_sigma=0.0):
    from synth import scene_sphere_box, cameras_on_sphere, make_ray_pool, prior_grid, sample_batch
    from synth import stratified_uniforms, random_colours, init_params

    a = orc.Arch(L=4, F=2, log2T=12, n_min=4, n_max=32, width=16, hidden=2, lambda_d=0.1,
                 lambda_sigma=lambda_sigma)
    sc = scene_sphere_box()
    pool = make_ray_pool(sc, cameras_on_sphere(4, 2.0, 40, 32, 32, 0), 256, 0)
    rays = sample_batch(pool, 6, 1)
    rays["is_obj"][:2] = 0  # keep some background rays in the batch
    grid = prior_grid(sc, 16, 0)
    nr, nc = 8, 16
    u = stratified_uniforms(6, nr, 2)
    cr = random_colours(6, 3)
    theta = init_params(orc.n_hash_params(a), a.mlp_shapes(), 4, hash_range=0.5).astype(np.float64)
    return a, theta, grid, rays, nc, nr, u, cr


def _fd4(f, theta, i):
    """Fourth-order central difference; its roundoff is ~eps |L| / h = 1e-12 here."""
    h = 1e-4 * max(1.0, abs(theta[i]))
    vals = []
    for s in (-2, -1, 1, 2):
        tp = theta.copy()
        tp[i] += s * h
        vals.append(f(tp))
    return (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)


def _check_fd(f, theta, g, idx):
    scale = np.abs(g[idx]).max()
    assert scale > 0
    bad = []
    for i in idx:
        fd = _fd4(f, theta, i)
        if abs(fd - g[i]) > 1e-6 * abs(g[i]) + 1e-9 * scale:
            bad.append((int(i), fd, g[i]))
    assert not bad, bad


@pytest.mark.parametrize("lambda_sigma", [0.0, 1e-2])
def test_gradient_matches_central_differences(orc, lambda_sigma):
    a, theta, grid, rays, nc, nr, u, cr = _fd_setup(orc, lambda_sigma)
    out = orc.batch(a, theta, grid, rays, nc, nr, u=u, c_rand=cr, want_grad=True)
    g = out["grad"]
    rng = np.random.default_rng(9)
    nh = orc.n_hash_params(a)
    touched = np.nonzero(g[:nh])[0]
    idx = np.concatenate([rng.choice(touched, 40, replace=False), nh + rng.choice(g.size - nh, 40, replace=False)])
    _check_fd(lambda tt: orc.batch(a, tt, grid, rays, nc, nr, u=u, c_rand=cr, want_samples=False)["loss"],
              theta, g, idx)


def test_upstream_gradient_matches_central_differences(orc):
    a, theta, grid, rays, nc, nr, u, cr = _fd_setup(orc)
    up = np.random.default_rng(10).normal(size=(6, 5))
    out = orc.batch(a, theta, grid, rays, nc, nr, u=u, upstream=up, want_grad=True)
    # the upstream functional equals sum_r up_r . (C_r, D_r, A_r)
    lin = np.sum(up[:, :3] * out["rgb"]) + up[:, 3] @ out["depth"] + up[:, 4] @ out["acc"]
    assert abs(lin - out["loss"]) < 1e-12
    g = out["grad"]
    nh = orc.n_hash_params(a)
    idx = np.concatenate([np.nonzero(g[:nh])[0][:30], np.arange(nh, nh + 30)])
    _check_fd(lambda tt: orc.batch(a, tt, grid, rays, nc, nr, u=u, upstream=up, want_samples=False)["loss"],
              theta, g, idx)


def test_sampler_does_not_depend_on_theta(orc):
    a, theta, grid, rays, nc, nr, u, cr = _fd_setup(orc)
    o1 = orc.batch(a, theta, grid, rays, nc, nr, u=u, c_rand=cr)
    o2 = orc.batch(a, theta * 3.0, grid, rays, nc, nr, u=u, c_rand=cr)
    np.testing.assert_array_equal(o1["t"], o2["t"])
    np.testing.assert_array_equal(o1["bins"], o2["bins"])


# ------------------------------------------------------------------------ Adam
def test_adam_constant_gradient_steps(orc):
    n = 7
    g = np.array([3.0, -2.0, 1e-3, -1e-6, 5.0, -7.0, 0.0])
    theta = np.zeros(n)
    m = np.zeros(n)
    v = np.zeros(n)
    lr = 1e-2
    for step in (1, 2, 3):
        before = theta.copy()
        orc.adam(theta, m, v, g, step, lr, 0.9, 0.99, 1e-15)
        # bias-corrected moments of a constant gradient are g and g^2, so each step is
        # -lr g / (|g| + eps): lr sign(g) up to the eps term (visible at |g| = 1e-6)
        np.testing.assert_allclose(theta - before, -lr * g / (np.abs(g) + 1e-15), rtol=1e-12, atol=0)


# ---------------------------------------------------------------------- Philox
def test_philox_known_answers(orc):
    # Known-answer vectors of Philox4x32-10 published with the Random123 library
    assert orc.philox4x32_10([0, 0, 0, 0], [0, 0]).tolist() == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert orc.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2).tolist() == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert orc.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]).tolist() == [
        0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_philox_uniforms_are_stratified(orc):
    nr = 48
    u = orc.philox_uniforms(1234, 3, 1, 200, nr)
    k = np.arange(nr)
    assert np.all(u >= k / nr) and np.all(u < (k + 1) / nr)
    c = orc.philox_colours(1234, 3, 1, 5000)
    assert c.min() >= 0 and c.max() < 1 and abs(c.mean() - 0.5) < 0.01


# ------------------------------------------------------------------ Reptile (§III-A, Eq. 2)
def test_reptile_special_cases(orc):
    theta = np.array([1.0, -2.0, 0.5, 8.0])
    t1 = np.array([3.0, 2.0, 0.5, -8.0])
    # beta = 0 leaves the meta-parameters alone; one task with beta = 1 copies it
    x = theta.copy()
    orc.reptile(x, [t1], 0.0)
    np.testing.assert_array_equal(x, theta)
    x = theta.copy()
    orc.reptile(x, [t1], 1.0)
    np.testing.assert_array_equal(x, t1)
    # one task, beta = 1/4: theta + (t - theta)/4 (dyadic, so exact)
    x = theta.copy()
    orc.reptile(x, [t1], 0.25)
    np.testing.assert_array_equal(x, np.array([1.5, -1.0, 0.5, 4.0]))
    # tasks symmetric about theta cancel; beta = 1 lands on the mean of the tasks
    x = theta.copy()
    orc.reptile(x, [theta + 1.0, theta - 1.0, theta + 0.5, theta - 0.5], 0.7)
    np.testing.assert_array_equal(x, theta)
    x = theta.copy()
    orc.reptile(x, [np.zeros(4), np.full(4, 2.0), np.full(4, 4.0), np.full(4, 6.0)], 1.0)
    np.testing.assert_array_equal(x, np.full(4, 3.0))


def test_reptile_is_the_mean_step_and_order_free(orc):
    rng = np.random.default_rng(5)
    theta = rng.normal(size=1000)
    tasks = [rng.normal(size=1000) for _ in range(16)]
    a = theta.copy()
    orc.reptile(a, tasks, 0.1)
    b = theta.copy()
    orc.reptile(b, tasks[::-1], 0.1)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)
    # n tasks at once = one task equal to their mean (Eq. 2 with theta_i^(q) the mean)
    c = theta.copy()
    orc.reptile(c, [np.mean(tasks, axis=0)], 0.1)
    np.testing.assert_allclose(a, c, rtol=0, atol=1e-14)
    # two half steps toward a fixed target compose to one step of 1 - (1 - beta)^2
    d = theta.copy()
    orc.reptile(d, [tasks[0]], 0.5)
    orc.reptile(d, [tasks[0]], 0.5)
    e = theta.copy()
    orc.reptile(e, [tasks[0]], 0.75)
    np.testing.assert_allclose(d, e, rtol=0, atol=1e-14)


def test_meta_step_composes_inner_training_and_outer_update(orc):
    """The meta-step driver: no inner steps leaves theta unchanged; one task with
    beta = 1 yields exactly that task trained alone from theta (Eq. 1 then Eq. 2)."""
    from helpers import CFG1, case

    a, theta, grid, rays, u, cr = case(CFG1, 16, 8, 8, seed=3, hash_range=0.5)
    b = dict(rays, u=u, c_rand=cr)
    th, losses = orc.meta_step(a, theta, lambda t: grid, [[], []], 8, 8, beta=0.5)
    np.testing.assert_array_equal(th, theta.astype(np.float64))
    th, losses = orc.meta_step(a, theta, lambda t: grid, [[b, b]], 8, 8, lr=1e-2, beta=1.0)
    ob = orc.OracleObject(a, theta, grid)
    l0 = ob.train_step(rays, 8, 8, u=u, c_rand=cr, lr=1e-2)
    l1 = ob.train_step(rays, 8, 8, u=u, c_rand=cr, lr=1e-2)
    # theta + 1 (x - theta) equals x up to one rounding of the subtraction and the sum
    np.testing.assert_allclose(th, ob.theta, rtol=0, atol=4 * np.finfo(np.float64).eps * np.abs(ob.theta).max())
    assert losses == [[l0, l1]] and l1 < l0


# ------------------------------------------------------------- prior grid refresh and Eq. 3
def _affine_field_arch(orc):
    # two dense levels (N = 4, 8: (N+1)^3 <= 2^12), one hidden layer of 16
    return orc.Arch(L=2, F=2, log2T=12, n_min=4, n_max=8, width=16, hidden=1, lambda_d=0.1, lambda_sigma=0.0)


def test_density_grid_closed_forms(orc):
    a = _affine_field_arch(orc)
    theta = np.zeros(orc.param_count(a))
    R = 6
    # zero output weights: o_0 = 0, sigma = 1 everywhere
    np.testing.assert_array_equal(orc.density_grid(a, theta, R), np.ones((R, R, R)))
    # features affine in the vertex position (reproduced exactly by trilinear
    # interpolation), positive so ReLU passes them: level 0 = (1+x, 1+y),
    # level 1 = (1+z, 1); hidden units copy the first three features; o_0 mixes them
    for l in range(2):
        N = orc.level_res(a, l)
        off = orc.level_offset(a, l)
        for cz in range(N + 1):
            for cy in range(N + 1):
                for cx in range(N + 1):
                    e = orc.grid_index(a, l, cx, cy, cz)
                    f = (1 + cx / N, 1 + cy / N) if l == 0 else (1 + cz / N, 1.0)
                    theta[off + 2 * e: off + 2 * e + 2] = f
    w1 = orc.mlp_offset(a, 0)
    for h in range(3):
        theta[w1 + h * 4 + h] = 1.0  # W_1 [16][4]: h0 = e0, h1 = e1, h2 = e2
    wo = orc.mlp_offset(a, 1)
    theta[wo: wo + 3] = [0.5, 0.25, 0.125]  # row 0 of W_out [4][16]
    g = orc.density_grid(a, theta, R)
    c = (np.arange(R) + 0.5) / R
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    np.testing.assert_allclose(g, np.exp(0.5 * (1 + x) + 0.25 * (1 + y) + 0.125 * (1 + z)), rtol=1e-13)


def _l_shape(n=600, seed=0):
    """Points of an L with unequal arms in the x-y plane (no rotational symmetry), z in [-0.2, 0.2]."""
    rng = np.random.default_rng(seed)
    a = np.c_[rng.uniform(-0.5, 0.5, n // 2), rng.uniform(-0.5, -0.3, n // 2)]  # long arm along x
    b = np.c_[rng.uniform(-0.5, -0.3, n // 2), rng.uniform(-0.3, 0.2, n // 2)]  # short arm along y
    xy = np.r_[a, b]
    return np.c_[xy, rng.uniform(-0.2, 0.2, xy.shape[0])]


def _splat(P, R):
    """Density grid of a cloud already in [0,1]^3: points per voxel (a prior of that exact pose)."""
    g = np.zeros((R, R, R))
    idx = np.clip((P * R).astype(int), 0, R - 1)
    np.add.at(g, (idx[:, 2], idx[:, 1], idx[:, 0]), 1.0)
    return g


def _normalise(P):
    lo, hi = P.min(0), P.max(0)
    return (P - 0.5 * (lo + hi)) / (hi - lo) + 0.5


def test_canonical_yaw_recovers_the_prior_pose(orc):
    P = _l_shape()
    grid = _splat(_normalise(P), 16)
    n_gamma = 36
    # a constant prior scores every yaw alike: c x |P|
    best, score = orc.canonical_yaw(np.full((8, 8, 8), 2.5), P, n_gamma)
    assert best == 0
    np.testing.assert_allclose(score, 2.5 * P.shape[0], rtol=1e-13)
    for g0 in (0, 5, 13, 27):
        ang = -2 * np.pi * g0 / n_gamma  # the observed cloud is the canonical one turned by -gamma_g0
        c, s = np.cos(ang), np.sin(ang)
        Q = P @ np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]]).T
        best, score = orc.canonical_yaw(grid, Q, n_gamma)
        assert best == g0, (g0, best)
        # turning the cloud by one more yaw step shifts the scores by one sample
        c1, s1 = np.cos(-2 * np.pi / n_gamma), np.sin(-2 * np.pi / n_gamma)
        Q1 = Q @ np.array([[c1, -s1, 0], [s1, c1, 0], [0, 0, 1]]).T
        _, score1 = orc.canonical_yaw(grid, Q1, n_gamma)
        np.testing.assert_allclose(score1, np.roll(score, 1), rtol=1e-9, atol=1e-9 * score.max())


# ------------------------------------------------------------ training rays (§III-B "Training Data")
def _kf_scene(seed=3, H=90, W=120, n_kf=2, yaw=0.7):
    import synth

    sc = synth.scene_random_csg(seed)
    obj = synth.object_pose([1.0, 2.0, 0.4], yaw, [0.6, 0.5, 0.4])
    kfs = [synth.render_keyframe(sc, p, obj, H, W, 50, 7) for p in synth.keyframe_cameras(n_kf, obj[1], 2.0, seed)]
    state = dict(instance=7, R_wo=obj[0], centre=obj[1], size=obj[2])
    return sc, obj, kfs, state


def test_rays_identity_pose_and_principal_ray(orc):
    H, W = 9, 11
    kf = dict(rgb=np.full((H, W, 3), 51, np.uint8), depth=np.full((H, W), 2.25, np.float32),
              mask=np.full((H, W), 3, np.int32), fx=100.0, fy=100.0, cx=5.5, cy=4.5,
              R_wc=np.eye(3), t_wc=np.array([0.5, 0.5, -2.0]))
    state = dict(instance=3, R_wo=np.eye(3), centre=[0.5, 0.5, 0.5], size=[1.0, 1.0, 1.0])
    # pixel (5, 4) has its centre on the principal point: the ray is the camera axis
    count = H * W
    draw = np.array([int(((4 * W + 5) << 32) // count) + 1], np.uint32)  # the candidate index 4 W + 5
    rays, n = orc.make_rays([kf], state, draw)
    assert n == count  # every pixel's ray meets the unit cube 2 units away (offsets <= 2 x 0.055)
    np.testing.assert_array_equal(rays["o"][0], [0.5, 0.5, -2.0])
    np.testing.assert_array_equal(rays["d"][0], [0.0, 0.0, 1.0])
    assert rays["depth"][0] == np.float32(2.25) and rays["is_obj"][0] == 1
    np.testing.assert_array_equal(rays["rgb"][0], np.float32(51) / np.float32(255))
    # the first and the last candidate are reached by the extreme draws
    rays, _ = orc.make_rays([kf], state, np.array([0, 2 ** 32 - 1], np.uint32))
    np.testing.assert_allclose(rays["d"][0], np.array([-5.0, -4.0, 100.0]) / np.sqrt(10041.0), rtol=1e-6)
    np.testing.assert_allclose(rays["d"][1], np.array([5.0, 4.0, 100.0]) / np.sqrt(10041.0), rtol=1e-6)
    # nothing in front of the camera: no candidate, the null ray
    kf2 = dict(kf, t_wc=np.array([0.5, 0.5, 3.0]))
    rays, n = orc.make_rays([kf2], state, np.array([7], np.uint32))
    assert n == 0 and np.all(rays["o"][0] == -1) and np.all(rays["d"][0] == 0) and rays["is_obj"][0] == 0


def test_rays_depth_target_lands_on_the_surface(orc):
    """o + depth d of an object ray is the rendered surface point in the object
    frame; every object pixel with depth is a candidate; background rays meet the box."""
    sc, obj, kfs, state = _kf_scene()
    rng = np.random.default_rng(0)
    draws = rng.integers(0, 2 ** 32, 4000, dtype=np.uint64).astype(np.uint32)
    rays, n = orc.make_rays(kfs, state, draws)
    n_obj_pixels = sum(int((k["mask"] == 7).sum()) for k in kfs)
    assert n_obj_pixels > 100 and n > n_obj_pixels
    m = rays["is_obj"] == 1
    assert 0 < m.sum() < len(m)
    p = rays["o"][m].astype(np.float64) + rays["depth"][m, None] * rays["d"][m].astype(np.float64)
    assert np.all(np.abs(sc.sdf(p)) < 2e-4)  # on the union's surface (FP32 inputs)
    # background rays enter the unit cube (the box) and miss the shape
    from synth.scenes import _hits_unit_cube

    assert np.mean(_hits_unit_cube(rays["o"][~m].astype(np.float64), rays["d"][~m].astype(np.float64))) > 0.99
    # the candidate count agrees with an FP64 count of box-hitting pixels up to grazing rays
    brute = 0
    for k in kfs:
        H, W = k["depth"].shape
        ys, xs = np.mgrid[0:H, 0:W]
        dc = np.stack([(xs + 0.5 - k["cx"]) / k["fx"], (ys + 0.5 - k["cy"]) / k["fy"], np.ones((H, W))], -1)
        dw = dc.reshape(-1, 3) @ np.asarray(k["R_wc"], np.float64).T
        dh = dw / np.linalg.norm(dw, axis=1, keepdims=True)
        R, c, S = obj
        o_n = ((np.asarray(k["t_wc"], np.float64) - c) @ R) / S + 0.5
        d_n = (dh @ R) / S
        brute += int(_hits_unit_cube(np.broadcast_to(o_n, d_n.shape), d_n).sum())
    assert abs(n - brute) <= 0.002 * brute + 4
