"""Host check that the tensor-core sweeps' pipeline cannot deadlock.

The kernel (csrc/band_tc.cu) runs a TMA producer, one MMA issuer and per TMEM
lane quarter one or two worker warps, handing buffers over by mbarriers: a
staging ring of planes, an A-operand ring in tensor memory (a slot freed by
the issuer's commit after the last products that read it), and accumulator
slots (freed when a worker has read its output).  Each role waits in a fixed
order, so whether the pipeline can stall for good depends only on those
orders and the ring sizes.  This module replays the waits of every role on a
model of the buffers, with the constants the library reports for each
(shape, radius, path) (mms_tc_pipeline_config), over tile sequences with
ragged and one-plane z chunks, and requires every output to drain.  The model
itself is pinned by configurations one step past the bounds, which must
stall.
"""
import pytest

import paper_2507_11067_gb300 as mms

LAYOUTS = [[64], [64, 64, 11], [16] * 5 + [3], [1], [2, 1], [1, 1, 1], [3, 64, 1], [40, 40, 40, 7], [5, 6]]


def simulate(mode, R, cfg, tiles):
    """True if every output of the tiles (their z-chunk lengths) drains."""
    PR, NST, ND = cfg["a_ring"], cfg["staging"], cfg["accumulators"]
    LOOK, mixed, ndrain = cfg["look"], bool(cfg["mixed"]), cfg["drainers"]
    reach = cfg["reach"]
    RZ = cfg["z_halo"]
    plane_tile, outs = [], []          # per global plane: (kb, jb, p, nzt); per output: (kb, z, nzt)
    kb = jb = 0
    for nzt in tiles:
        for p in range(nzt + 2 * RZ):
            plane_tile.append((kb, jb, p, nzt))
        for z in range(nzt):
            outs.append((kb, z, nzt))
        kb += nzt + 2 * RZ
        jb += nzt
    K, J = len(plane_tile), len(outs)
    need = [kbo + z + reach for kbo, z, _ in outs]
    # the output whose products' commit frees each plane's A slot
    freed_by = [None] * K
    for j, (kbo, z, nzt) in enumerate(outs):
        if mode == "star":
            if z == 0:
                for p in range(R):
                    freed_by[kbo + p] = j
            freed_by[kbo + z + R] = j
            if z == nzt - 1:
                for p in range(nzt + R, nzt + 2 * R):
                    freed_by[kbo + p] = j
        else:
            freed_by[kbo + z] = j
            if mode == "box" and z == nzt - 1:
                for p in range(nzt, nzt + 2 * R):
                    freed_by[kbo + p] = j
    assert all(f is not None for f in freed_by)
    loaded, conv, issued, drained = [False] * K, [False] * K, [False] * J, [False] * J

    def can_convert(k):
        if not loaded[k]:
            return False
        if k >= PR and not issued[freed_by[k - PR]]:
            return False
        if mode == "star":   # the plane that completes output zo writes its z sum beside the accumulator
            kbp, jbp, p, nzt = plane_tile[k]
            zo = p - 2 * R
            if 0 <= zo < nzt and jbp + zo >= ND and not drained[jbp + zo - ND]:
                return False
        return True

    if mixed:
        workers = [["mix", w, w] for w in range(2)]           # kind, next plane, next output
    else:
        workers = [["conv", 0]] + [["drain", e] for e in range(ndrain)]
    nload = nissue = 0
    moved = True
    while moved:
        moved = False
        if nload < K and (nload < NST or conv[nload - NST]):
            loaded[nload] = True
            nload += 1
            moved = True
        if nissue < J:
            j = nissue
            if all(conv[: need[j] + 1]) and (j < ND or drained[j - ND]):
                issued[j] = True
                nissue += 1
                moved = True
        for wk in workers:
            if wk[0] == "mix":
                kc, jd = wk[1], wk[2]
                if kc < K and (jd >= J or kc <= need[jd] + LOOK):
                    if can_convert(kc):
                        conv[kc] = True
                        wk[1] += 2
                        moved = True
                elif jd < J and issued[jd]:
                    drained[jd] = True
                    wk[2] += 2
                    moved = True
            elif wk[0] == "conv":
                if wk[1] < K and can_convert(wk[1]):
                    conv[wk[1]] = True
                    wk[1] += 1
                    moved = True
            else:
                if wk[1] < J and issued[wk[1]]:
                    drained[wk[1]] = True
                    wk[1] += ndrain
                    moved = True
    return all(drained)


def library_configs():
    out = []
    for shape, mode in (("box", "box"), ("star", "star"), ("box2d", "planar")):
        for r in (1, 2, 3, 4):
            for path in ("bf16x3", "3xtf32", "tf32"):
                cfg = mms.tc_pipeline_config(shape, r, path)
                if cfg is not None:
                    out.append((shape, mode, r, path, cfg))
    return out


def test_every_configuration_is_reported():
    cfgs = library_configs()
    assert len(cfgs) == 36
    assert mms.tc_pipeline_config("box", 5, "bf16x3") is None
    assert mms.tc_pipeline_config("box", 2, "cuda_core") is None


@pytest.mark.parametrize("shape,mode,r,path,cfg", library_configs(),
                         ids=lambda v: v if isinstance(v, (str, int)) else None)
def test_library_pipeline_drains(shape, mode, r, path, cfg):
    # the star keeps its z sums in one converter's registers: never mixed
    if mode == "star":
        assert not cfg["mixed"]
    if cfg["mixed"]:
        assert cfg["accumulators"] == 2 and cfg["a_ring"] % 2 == 0 and cfg["staging"] % 2 == 0
    for tiles in LAYOUTS:
        assert simulate(mode, r, cfg, tiles), (shape, r, path, cfg, tiles)


def _mixed_box(R, PR, LOOK):
    return {"a_ring": PR, "staging": 8, "accumulators": 2, "look": LOOK, "mixed": 1, "drainers": 2,
            "reach": 2 * R, "z_halo": R}


def test_model_mixed_lookahead_bound():
    # a mixed worker may convert up to PR - reach + 1 planes past its next
    # output's last plane: the slot it waits for is freed by products that
    # need its own drain of the output two before, which it has done; one
    # more plane and that drain comes after the wait
    for R, PR in ((1, 10), (2, 8), (3, 8)):
        edge = PR - 2 * R + 1
        assert all(simulate("box", R, _mixed_box(R, PR, edge), t) for t in LAYOUTS)
        assert not all(simulate("box", R, _mixed_box(R, PR, edge + 1), t) for t in LAYOUTS)


def test_model_star_ring_bound():
    # a star tile's first output waits for its first 2r+1 planes, all in the
    # A ring at once: a ring of 2r planes stalls at the first tile
    for R in (1, 2, 3, 4):
        cfg = {"a_ring": 2 * R + 1, "staging": max(8, 2 * R + 2), "accumulators": 1, "look": 0, "mixed": 0,
               "drainers": 1, "reach": 2 * R, "z_halo": R}
        assert all(simulate("star", R, cfg, t) for t in LAYOUTS)
        cfg["a_ring"] = 2 * R
        assert not simulate("star", R, cfg, [8])
