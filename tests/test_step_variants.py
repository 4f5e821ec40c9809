"""Per-step tile variants on the host (no GPU): which variants a step offers,
what choosing one changes in the launch list, and the errors."""
import pytest

import circuit_inputs as ci

ST_PERMUTE, ST_BPREP_TC, ST_GEMM_TC = 1, 2, 3


@pytest.fixture(scope="module")
def tn():
    import paper_2111_03011_gb300 as m
    return m


@pytest.fixture(scope="module")
def plan30(tn):
    cfg = ci.config_sliced30()
    return tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_only=True, gemm=4,
                      order_trials=2048)


def _tile(s, cap, pair):
    """(BN, fold, paired) of a tensor-core GEMM step under (cap, pair), by the
    rule the kernel dispatch states: widest power of two <= cap covering 2N,
    or patterns sharing A folded side by side up to cap columns."""
    n2 = 2 << s["nn"]
    w, fold = n2, 1
    if s["mapA"][0] == 1 and s["PC"] > 1 and 16 <= n2 < cap:
        while w < cap and fold < s["PC"]:
            w, fold = 2 * w, 2 * fold
    bn = 16
    while bn < 256 and bn < min(w, cap):
        bn *= 2
    return bn, fold, s["h16"] != 0 and bn == 256 and (1 << s["nm"]) >= 256 and pair >= 0


def test_variant_counts_and_defaults(tn, plan30):
    d = tn.tn_plan_describe(plan30)
    n_gemm_multi = n_perm_multi = n_bprep_multi = 0
    for i, s in enumerate(d["steps"]):
        n, chosen = tn.tn_plan_step_variants(plan30, i)
        assert chosen == 0 and s["variant"] == 0
        if s["kind"] == ST_GEMM_TC:
            distinct = {_tile(s, c, p) for c, p in ((256, 0), (256, -1), (128, 0), (64, 0), (32, 0))}
            assert n == len(distinct)
            assert (s["tile_cap"], s["pair"]) == (256, 0)
            n_gemm_multi += n > 1
        elif s["kind"] == ST_PERMUTE:
            assert n == len(s["alts"]) >= 1
            if (s["PA"] << s["rA"]) < 1 << 20:
                assert n == 1
            assert (s["t_bits"], s["n_rest"], s["tab_off"]) == (
                s["alts"][0]["t_bits"], s["alts"][0]["n_rest"], s["alts"][0]["tab_off"])
            n_perm_multi += n > 1
            assert s["alts"][0]["vec4"] == 0 and all(
                b["vec4"] == 1 and b["tab_off"] == a["tab_off"] for a, b in zip(s["alts"], s["alts"][1:]) if b["vec4"])
        elif s["kind"] == ST_BPREP_TC:
            assert n == (2 if s["alts"] else 1)
            n_bprep_multi += n > 1
        else:
            assert n == 1
    # the 30-qubit plan has tunable GEMM tiles, permute schedules and B preparations
    assert n_gemm_multi >= 5 and n_perm_multi >= 3 and n_bprep_multi >= 1
    assert tn.tn_plan_get_stats(plan30)["n_tuned_steps"] == 0


def test_choosing_a_variant_changes_only_its_launch(tn):
    cfg = ci.config_sliced30()
    p = tn.tn_plan(cfg["circuit"], cfg["open_qubits"], cfg["tails"], cfg["edges"], host_only=True, gemm=4,
                   order_trials=2048)
    d0 = tn.tn_plan_describe(p)
    caps = [(256, 0), (256, -1), (128, 0), (64, 0), (32, 0)]
    for i, s in enumerate(d0["steps"]):
        n, _ = tn.tn_plan_step_variants(p, i)
        for v in range(n):
            tn.tn_plan_set_step_variant(p, i, v)
            x = tn.tn_plan_describe(p)["steps"][i]
            assert x["variant"] == v and tn.tn_plan_step_variants(p, i) == (n, v)
            if s["kind"] == ST_PERMUTE:
                a = s["alts"][v]
                assert (x["t_bits"], x["tab_off"], x["n_rest"], x["rest_in"], x["rest_out"], x["vec4"]) == (
                    a["t_bits"], a["tab_off"], a["n_rest"], a["rest_in"], a["rest_out"], a["vec4"])
            elif s["kind"] == ST_GEMM_TC:
                # the v-th distinct tile of the list, in list order
                seen, picks = [], []
                for c in caps:
                    t = _tile(s, *c)
                    if t not in seen:
                        seen.append(t)
                        picks.append(c)
                assert (x["tile_cap"], x["pair"]) == picks[v]
        with pytest.raises(tn.TNError):
            tn.tn_plan_set_step_variant(p, i, n)
        with pytest.raises(tn.TNError):
            tn.tn_plan_set_step_variant(p, i, -1)
    st = tn.tn_plan_get_stats(p)
    d1 = tn.tn_plan_describe(p)
    assert st["n_tuned_steps"] == sum(s["variant"] != 0 for s in d1["steps"])
    # everything but the variant fields is unchanged
    for s0, s1 in zip(d0["steps"], d1["steps"]):
        for k in s0:
            if k not in ("variant", "tile_cap", "pair", "t_bits", "tab_off", "n_rest", "rest_in", "rest_out",
                         "vec4"):
                assert s0[k] == s1[k], k
    with pytest.raises(tn.TNError):
        tn.tn_plan_step_variants(p, len(d0["steps"]))
    with pytest.raises(tn.TNError):
        tn.tn_plan_tune_steps(p)          # host-only plan: no device to time on
