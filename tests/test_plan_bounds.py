"""Every launch of a plan stays inside the memory it is given (CPU, no GPU).

For each step of the plan's launch list (from tn_plan_describe), the bytes
each kernel reads and writes -- as the kernels index them: pattern strides,
split planes, real embeddings, gather tables -- must lie inside the workspace
buffer or leaf variant it is handed, every table index inside the meta
buffer, and buffers that are live at the same time must not overlap.  A
launch that wrote past its buffer (for example a split permute writing two
operand planes into space sized for one) fails here before it ever runs on a
GPU.
"""
import numpy as np
import pytest

import circuit_inputs as ci


@pytest.fixture(scope="module")
def tn():
    import paper_2111_03011_gb300 as m
    return m


ST_SMALL, ST_PERMUTE, ST_BPREP_TC, ST_GEMM_TC, ST_BPREP_C, ST_GEMM_SIMT, ST_ABSMAX = range(7)


def _perm_bit_map(meta, sc, r):
    """Output bit position of every input bit under one permute schedule, as
    the kernel indexes it: out[bo + out_off[j]] = in[bi + in_off[slot[j]]]
    inside a tile, the remaining bits moved by rest_in -> rest_out.  Also
    checks that the three tables are OR-linear in the tile index (so the
    single-bit images fix the whole map) and stay inside the tensor."""
    t = sc["t_bits"]
    nt = 1 << t
    assert t + sc["n_rest"] == r and sc["n_rest"] <= 32 and t <= 10
    assert sc["tab_off"] + 3 * nt <= meta.size
    tab = meta[sc["tab_off"]:sc["tab_off"] + 3 * nt]
    assert (tab >= 0).all() and (tab < (1 << r)).all()
    s_in, s_out, slot = tab[:nt], tab[nt:2 * nt], tab[2 * nt:]
    assert (slot < nt).all()
    if sc["vec4"]:      # outputs 4g .. 4g + 3 of a tile are consecutive, from a 4-aligned offset
        assert t >= 2 and s_out[1] == 1 and s_out[2] == 2
        assert all(x >= 2 for x in sc["rest_out"])
    img = {}
    for u in range(t):
        j = 1 << u
        src, dst = int(s_in[slot[j]]), int(s_out[j])
        assert src & (src - 1) == 0 and dst & (dst - 1) == 0 and src and dst
        img[src.bit_length() - 1] = dst.bit_length() - 1
    js = np.arange(nt)
    for name, tb in (("out", s_out), ("slot", slot), ("in", s_in)):
        acc = np.zeros(nt, dtype=np.int64)
        for u in range(t):
            acc |= np.where((js >> u) & 1, tb[1 << u], 0)
        assert (acc == tb).all(), name
    assert (s_in[slot] == np.bitwise_or.reduce([np.where((js >> u) & 1, s_in[slot[1 << u]], 0)
                                                for u in range(t)] or [np.zeros(nt, np.int64)])).all()
    for a, b in zip(sc["rest_in"], sc["rest_out"]):
        assert 0 <= a < r and 0 <= b < r and a not in img
        img[a] = b
    assert sorted(img) == list(range(r))
    return [img[x] for x in range(r)]


def _check_plan(d):
    meta = np.asarray(d["meta"], dtype=np.int64)
    bufs = d["bufs"]
    ws = d["workspace_bytes"]
    leaf_info = d["leaf_info"]
    for off, nbytes, first, last in bufs:
        assert 0 <= off and off + nbytes <= ws
    for i, (o1, b1, f1, l1) in enumerate(bufs):           # live at the same time -> disjoint
        for (o2, b2, f2, l2) in bufs[i + 1:]:
            if f1 <= l2 and f2 <= l1:
                assert o1 + b1 <= o2 or o2 + b2 <= o1
    for off, size, nvar in leaf_info:
        assert off + size * (1 << nvar) <= d["leaf_arena_elems"]

    def cap(ref):
        """bytes available behind an operand reference"""
        kind, rid = ref
        return 8 * leaf_info[rid][1] if kind == 0 else bufs[rid][1]

    def table(mode, off, n, bound):
        """largest pattern index a map of `n` entries yields (mode 0 identity, 1 zero, 2 table)"""
        if mode == 0:
            return n - 1
        if mode == 1:
            return 0
        assert off + n <= meta.size
        t = meta[off:off + n]
        assert (t >= 0).all() and (t < bound).all()
        return int(t.max())

    for i, s in enumerate(d["steps"]):
        k = s["kind"]
        if k == ST_SMALL:
            pa = table(*s["mapA"], s["PC"], s["PA"])
            pb = table(*s["mapB"], s["PC"], s["PB"])
            assert 8 * (pa + 1) << s["rA"] <= cap(s["a"])
            assert 8 * (pb + 1) << s["rB"] <= cap(s["b"])
            assert 8 * s["PC"] << s["rC"] <= cap(s["c"])
            assert s["rA"] - s["nk"] + s["nn"] == s["rC"]
            assert all(0 <= x < s["rA"] for x in s["kposA"][:s["nk"]])
        elif k == ST_PERMUTE:
            n = s["PA"] << s["rA"]
            assert 8 * n <= cap(s["a"])
            per = {0: 8, 1: 16, 2: 8, 3: 8}[s["split"]]       # bytes written per complex element (both planes)
            assert per * n <= cap(s["c"]), (i, s["split"])
            # the chosen schedule and every alternative a tuner may pick: tables
            # inside meta, and each one the same bit permutation as the default
            scheds = [s] + list(s["alts"])
            assert s["alts"] and 0 <= s["variant"] < len(s["alts"])
            maps = [_perm_bit_map(meta, x, s["rA"]) for x in scheds]
            assert all(m == maps[1] for m in maps), i
            assert sorted(maps[0]) == list(range(s["rA"]))
        elif k in (ST_BPREP_TC, ST_BPREP_C):
            assert 8 * s["PA"] << s["rA"] <= cap(s["a"])
            K, N = 1 << s["nk"], 1 << s["nn"]
            assert s["bk_off"] + K <= meta.size and s["bn_off"] + N <= meta.size
            assert max(meta[s["bk_off"]:s["bk_off"] + K].max(), meta[s["bn_off"]:s["bn_off"] + N].max()) < (
                1 << s["rA"])
            if k == ST_BPREP_TC:
                es = 4 if s["h16"] == 0 else 2
                assert 2 * s["PA"] * (2 * N) * (2 * K) * es <= cap(s["c"])
                if s["alts"]:
                    # the permute alternative: K legs to output bits 0 .. nk-1, N legs
                    # above them (the order the gather tables encode); it writes
                    # the same embedded planes into the same buffer
                    bkt = meta[s["bk_off"]:s["bk_off"] + K]
                    bnt = meta[s["bn_off"]:s["bn_off"] + N]
                    want = {}
                    for q in range(s["nk"]):
                        want[int(bkt[1 << q]).bit_length() - 1] = q
                    for q in range(s["nn"]):
                        want[int(bnt[1 << q]).bit_length() - 1] = s["nk"] + q
                    assert s["rA"] == s["nk"] + s["nn"] and sorted(want) == list(range(s["rA"]))
                    assert _perm_bit_map(meta, s["alts"][0], s["rA"]) == [want[x] for x in range(s["rA"])]
                    assert not s["alts"][0]["vec4"] and s["fork"] < 0
                    assert s["bprep_embed0"] == int(s["nk"] >= 1 and bkt[1] != 1)
            else:
                assert 8 * s["PA"] * K * N <= cap(s["c"])
        elif k in (ST_GEMM_TC, ST_GEMM_SIMT):
            M, N, K = 1 << s["nm"], 1 << s["nn"], 1 << s["nk"]
            pa = table(*s["mapA"], s["PC"], s["PA"])
            pb = table(*s["mapB"], s["PC"], s["PB"])
            assert pa < s["PA"] and pb < s["PB"]
            if k == ST_GEMM_TC:
                es = 4 if s["h16"] == 0 else 2
                assert 2 * K * es >= 16                        # TMA row pitch
                assert 2 * s["PA"] * M * (2 * K) * es <= cap(s["a"])
                assert 2 * s["PB"] * (2 * N) * (2 * K) * es <= cap(s["b"])
            else:
                assert 8 * s["PA"] * M * K <= cap(s["a"])
                assert 8 * s["PB"] * K * N <= cap(s["b"])
            assert 8 * s["PC"] * M * N <= cap(s["c"])
        elif k == ST_ABSMAX:
            assert 8 * s["PA"] << s["rA"] <= cap(s["a"])
        else:
            raise AssertionError(f"unknown step kind {k}")
    # B-prep steps run on the side stream from their fork: the fork is an
    # earlier tensor-core GEMM, the operand is written before it, and both the
    # operand and the output are live from the fork to the consuming GEMM (so
    # the disjointness above keeps every concurrent step off their memory)
    steps = d["steps"]
    for i, s in enumerate(steps):
        f = s.get("fork", -1)
        if f < 0:
            continue
        assert s["kind"] == ST_BPREP_TC and 0 <= f < i and steps[f]["kind"] == ST_GEMM_TC
        g = steps[i + 1]
        assert g["kind"] == ST_GEMM_TC and g["b"] == s["c"]
        out = bufs[s["c"][1]]
        assert out[2] <= f and out[3] >= i + 1
        if s["a"][0] == 1:
            prod = [j for j in range(i) if steps[j]["c"] == s["a"]]
            assert len(prod) == 1 and prod[0] < f
            assert bufs[s["a"][1]][2] <= prod[0] and bufs[s["a"][1]][3] >= i
            if s["slot"] >= 0:
                assert steps[prod[0]]["max_slot"] == s["slot"]
        else:
            assert s["slot"] < 0 or s["slot"] <= -2 or s["h16"] != 2
        assert all(steps[j]["c"] != s["a"] for j in range(f, i))
    f = d["final"]
    L = len(d.get("_tails", [])) or None
    assert 8 * f["PF"] << f["rF"] <= cap(f["ref"])
    assert all(0 <= x < f["rF"] for x in f["open_pos"])
    pidx = meta[f["pidx_off"]:f["pidx_off"] + (L or 1)]
    assert (pidx >= 0).all() and (pidx < f["PF"]).all()


CASES = [dict(r=3, c=4, m=6, seed=5, n_open=4, L=6, cut=1),
         dict(r=4, c=4, m=8, seed=11, n_open=6, L=8, cut=2),
         dict(r=2, c=4, m=8, seed=6, n_open=0, L=5, cut=1),
         dict(r=4, c=5, m=10, seed=13, n_open=8, L=24, cut=2),
         dict(r=3, c=5, m=12, seed=17, n_open=5, L=64, cut=3)]
ENGINES = [dict(gemm=1), dict(gemm=2), dict(gemm=3), dict(gemm=4), dict(gemm=4, small_max_bits=-1),
           dict(gemm=1, small_max_bits=-1), dict(gemm=4, small_max_bits=2)]


@pytest.mark.parametrize("case", CASES, ids=[f"{c['r']}x{c['c']}m{c['m']}L{c['L']}" for c in CASES])
def test_launch_extents_inside_buffers(tn, case):
    cfg = ci.config_small(case["r"], case["c"], case["m"], seed=case["seed"], n_open=case["n_open"], L=case["L"],
                          n_cut_gates=case["cut"])
    for eng in ENGINES:
        p = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_only=True, **eng)
        d = tn.tn_plan_describe(p, with_data=True)
        d["_tails"] = list(cfg["tails"])
        _check_plan(d)


def test_launch_extents_auto_sliced_and_random_gates(tn):
    cfg = ci.config_small(4, 5, 10, seed=13, n_open=8, L=24, n_cut_gates=1)
    for gemm in (1, 3, 4):
        p = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_only=True, gemm=gemm,
                       max_log2_elements=15, auto_slice=16)
        d = tn.tn_plan_describe(p, with_data=True)
        d["_tails"] = list(cfg["tails"])
        _check_plan(d)
    for seed in (1, 2, 3):
        c = ci.make_random_2q_circuit(10, 4, seed=seed)
        oq = [1, 4, 7]
        tails = ci.draw_tails(10, oq, 16, seed=seed)
        for gemm in (1, 4):
            p = tn.tn_plan(c, oq, tails, host_only=True, gemm=gemm, small_max_bits=-1)
            d = tn.tn_plan_describe(p, with_data=True)
            d["_tails"] = list(tails)
            _check_plan(d)


def test_launch_extents_of_the_30_qubit_workload(tn):
    cfg = ci.config_sliced30()
    for gemm in (1, 3, 4):
        p = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_only=True, gemm=gemm,
                       order_trials=2048, side_bprep=1)
        d = tn.tn_plan_describe(p, with_data=True)
        d["_tails"] = list(cfg["tails"])
        _check_plan(d)
        # the largest B-prep of the stem (an operand of 63 x 2^19 elements) runs beside a GEMM
        side = [s for s in d["steps"] if s.get("fork", -1) >= 0]
        assert tn.tn_plan_get_stats(p)["n_side_bprep"] == len(side) >= 1
        assert max(8 * s["PA"] << s["rA"] for s in side) >= 1 << 27
    p = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_only=True, gemm=4,
                   order_trials=2048)
    assert tn.tn_plan_get_stats(p)["n_side_bprep"] == 0
    assert all(s["fork"] == -1 for s in tn.tn_plan_describe(p)["steps"])
