"""Host-side executor of exported tile programmes (test code).

Runs the programme that ``sv_plan_export`` describes on a NumPy state, step
by step, following the documented meaning of each step (plan.h, tileprog.h),
in complex128.  Used to check the planner and the stage compiler against the
FP64 oracle without a GPU.  It shares no code with the oracle or the library.
"""
from __future__ import annotations

import numpy as np

TWO32 = 1 << 32
MASK32 = TWO32 - 1

# generic tile ops (plan.h)
TOP_GATE, TOP_GATE_CL, TOP_GATE_CG, TOP_DIAG, TOP_SWAP, TOP_H, TOP_X = range(7)
TERM_L, TERM_LL, TERM_G, TERM_LG, TERM_GG = range(5)
# register-stage ops (tileprog.h)
T2_STAGE, T2_GATE, T2_H, T2_X, T2_DIAG, T2_SCALE, T2_BLOCK, T2_RGATE, T2_ROT, T2_HPH, T2_HG = range(11)
C_NONE, C_REG, C_LANE, C_THREAD, C_GLOBAL = range(5)


def pdep(v: int, mask: int) -> int:
    r, b = 0, 0
    while mask:
        low = mask & -mask
        if (v >> b) & 1:
            r |= low
        mask &= mask - 1
        b += 1
    return r


def tile_index(p, base):
    k = p["k"]
    idx = np.full(1 << k, base, dtype=np.int64)
    loc = np.arange(1 << k)
    for s, q in enumerate(p["slot_phys"]):
        idx |= ((loc >> s) & 1) << q
    return idx


def mat_of(m):
    m = np.asarray(m, dtype=np.float64)
    return (m[0::2] + 1j * m[1::2]).reshape(2, 2)


def apply_pairs(t, bit, u, cond=None):
    loc = np.arange(t.size)
    sel = ((loc >> bit) & 1) == 0
    if cond is not None:
        sel &= cond
    i0 = loc[sel]
    i1 = i0 | (1 << bit)
    a, b = t[i0].copy(), t[i1].copy()
    t[i0] = u[0, 0] * a + u[0, 1] * b
    t[i1] = u[1, 0] * a + u[1, 1] * b


def phase_of(theta64):
    return np.exp(2j * np.pi * (theta64 / 2.0 ** 64))


def run_generic_pass(state, p):
    k = p["k"]
    ntiles = 1 << (int(np.log2(state.size)) - k)
    loc = np.arange(1 << k)
    for tile in range(ntiles):
        base = pdep(tile, p["gmask"])
        idx = tile_index(p, base)
        t = state[idx].copy()
        for op in p["ops"]:
            ty = op["type"]
            if ty == TOP_DIAG:
                phi = np.zeros(t.size, dtype=object)
                acc = np.zeros(t.size, dtype=np.float64)
                for kind, a, b, th in p["terms"][op["tb"]:op["te"]]:
                    if kind == TERM_L:
                        on = (loc >> a) & 1
                    elif kind == TERM_LL:
                        on = ((loc >> a) & 1) & ((loc >> b) & 1)
                    elif kind == TERM_G:
                        on = np.full(t.size, (base >> a) & 1)
                    elif kind == TERM_LG:
                        on = ((loc >> a) & 1) * ((base >> b) & 1)
                    else:
                        on = np.full(t.size, ((base >> a) & 1) & ((base >> b) & 1))
                    acc += on * (th / 2.0 ** 64)
                t *= np.exp(2j * np.pi * acc)
                del phi
            elif ty == TOP_SWAP:
                a, b = op["slot"], op["cslot"]
                sel = (((loc >> a) & 1) == 1) & (((loc >> b) & 1) == 0)
                i = loc[sel]
                j = i ^ (1 << a) ^ (1 << b)
                t[i], t[j] = t[j].copy(), t[i].copy()
            else:
                if ty == TOP_GATE_CG and not ((base >> op["cbit"]) & 1):
                    continue
                cond = None
                if ty == TOP_GATE_CL:
                    cond = ((loc >> op["cslot"]) & 1) == 1
                if ty == TOP_X:
                    u = np.array([[0, 1], [1, 0]], dtype=complex)
                elif ty == TOP_H:
                    u = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
                else:
                    u = mat_of(op["m"])
                apply_pairs(t, op["slot"], u, cond)
        state[idx] = t


def _expi32(u):
    return np.exp(2j * np.pi * ((u & MASK32) / 2.0 ** 32))


def run_t2_pass(state, p, t2=None, gen_basis=None, gen_h=0, bases=None):
    """Execute a register-stage pass.  `t2` defaults to the pass's programme;
    with `gen_basis` (a physical basis index) the pass starts from the product
    state H^{gen_h}|gen_basis> (H on the physical qubits of the mask gen_h)
    and generates its tiles instead of reading them (the programme is then the
    pass's generated-state variant, `t2gen`, whose own leading Hadamards on
    tile bits are unnormalised: its closing scale, `gen_scale`, which holds
    their 2^(-1/2), multiplies the generated state).
    `bases`: run only the tiles with these physical base indices, in order
    (default: every tile, in index order)."""
    t2 = t2 if t2 is not None else p["t2"]
    fmt = t2.get("format", 1)
    k = p["k"]
    ntiles = 1 << (int(np.log2(state.size)) - k)
    loc = np.arange(1 << k)
    stat = np.asarray(t2["stat"], dtype=np.int64)
    rb, nthreads = t2["rb"], t2["threads"]
    nw = nthreads.bit_length() - 1 - 5          # warp bits
    if fmt == 2:
        sc = np.asarray(t2["statc"], dtype=np.float64).reshape(-1, nthreads, 2)
        statc = sc[:, :, 0] + 1j * sc[:, :, 1]
    nstages = sum(1 for ins in t2["ins"] if ins["op"] == T2_STAGE)
    for base in (bases if bases is not None else (pdep(t_, p["gmask"]) for t_ in range(ntiles))):
        idx = tile_index(p, base)
        if gen_basis is None:
            t = state[idx].copy()
        else:  # the product state after the leading Hadamards
            # the programme's unnormalised leading Hadamards P on the recorded
            # H^{gen_h}|gen_basis>: H_unnorm H_norm = sqrt(2) I on a qubit in both
            P = t2["gen_hmask"]
            gl, hq_local = 0, 0
            for s_, q in enumerate(p["slot_phys"]):
                gl |= ((gen_basis >> q) & 1) << s_
                if (gen_h >> q) & 1:
                    hq_local |= 1 << s_
            hm = P ^ hq_local
            ghm = gen_h & p["gmask"]
            has = ((gen_basis ^ base) & p["gmask"] & ~ghm) == 0
            gneg = bin(base & gen_basis & ghm).count("1") & 1
            both = bin(P & hq_local).count("1")
            # the variant's closing scale is part of the generated state
            v = 2.0 ** (0.5 * (both - (bin(gen_h).count("1") - both))) * t2.get("gen_scale", 1.0)
            par = np.array([(bin(int(i) & gl & hm).count("1") + gneg) & 1 for i in loc])
            t = np.where(((loc ^ gl) & ~hm) == 0, np.where(par == 1, -v, v), 0.0).astype(complex)
            if not has:
                t[:] = 0
        lin = [0] * (16 * max(t2["nruns"], 1))
        cst = [0] * max(t2["nruns"], 1)
        for run, tb, g0, g1, th in t2["tterms"]:
            on = (base >> g0) & 1
            if g1 >= 0:
                on &= (base >> g1) & 1
            if on:
                if fmt == 2:
                    i = run * 16 + (tb if tb >= 0 else 15)
                    lin[i] = (lin[i] + th) & MASK32
                elif tb >= 0:
                    lin[run * 16 + tb] = (lin[run * 16 + tb] + th) & MASK32
                else:
                    cst[run] = (cst[run] + th) & MASK32
        if fmt == 2:
            slotv = [_expi32(lin[i0] + (lin[i1] if i1 >= 0 else 0)) for i0, i1 in t2["slots"]]
        st = None
        nst = 0
        for ins in t2["ins"]:
            op = ins["op"]
            if op == T2_STAGE:
                st = t2["stages"][ins["aux"]]
                reg, lane, warp = st[0:rb], st[5:10], st[10:10 + nw]
                assert sorted(reg + lane + warp) == list(range(k))
                assert reg[0] == 0
                if fmt == 1:
                    assert lane[:3] == [1, 2, 3]
                elif nst == 0 and gen_basis is None:
                    assert lane[:3] == [1, 2, 3]  # read in the bulk copies' linear order
                nst += 1
                if fmt == 2 and nst == nstages:
                    assert lane[:3] == [1, 2, 3]  # coalesced write-back
                ttb = lane + warp                   # tile bit of thread bit t
                tid = np.zeros(t.size, dtype=np.int64)
                for tt_, b in enumerate(ttb):
                    tid |= ((loc >> b) & 1) << tt_
                continue
            if op == T2_BLOCK:
                bl = np.asarray(t2["blocks"][ins["aux"]], dtype=np.float64)
                U = (bl[:1024] + 1j * bl[1024:]).reshape(32, 32)
                off = np.zeros(32, dtype=np.int64)
                for rho in range(32):
                    for j in range(5):
                        if (rho >> j) & 1:
                            off[rho] |= 1 << reg[j]
                regmask = int(off[31])
                bases = loc[(loc & regmask) == 0]
                X = t[bases[:, None] + off[None, :]]
                t[bases[:, None] + off[None, :]] = X @ U.T
                continue
            if op == T2_SCALE:
                m = t2["mats"][ins["aux"]]
                t *= np.float64(np.float32(m[0])) + np.float64(np.float32(m[1]))
                continue
            if op in (T2_DIAG, T2_HPH):  # T2_HPH: the run, then H on register bit idx
                facs = t2["fac2"] if fmt == 2 else t2["factors"]
                for f in facs[ins["e0"]:ins["e1"]]:
                    w0 = f["w0"]
                    if (w0 >> 28) & 1:  # 32-entry constant phase table (tileprog.h)
                        pb = (w0 >> 10) & 0xF
                        fl = np.asarray(t2["mats"][f["row"]:f["row"] + 8], dtype=np.float64).reshape(-1)
                        xs = np.arange(32)
                        tab = fl[4 * (xs >> 1) + (xs & 1)] + 1j * fl[4 * (xs >> 1) + 2 + (xs & 1)]
                        xr = np.zeros(t.size, dtype=np.int64)
                        for j in range(rb):
                            xr |= ((loc >> reg[j]) & 1) << j
                        fac = tab[xr]
                        if pb:
                            fac = np.where(((tid >> (pb - 1)) & 1) == 1, fac, 1.0)
                        t *= fac
                        continue
                    mask = w0 & 0xFF
                    sel = np.ones(t.size, dtype=bool)
                    for j in range(rb):
                        if (mask >> j) & 1:
                            sel &= ((loc >> reg[j]) & 1) == 1
                    dm = (w0 >> 19) & 0x1FF
                    if fmt == 2:  # static complex row x tile slot x one slot per dynamic bit
                        fac = statc[f["row"]][tid] if f["row"] >= 0 else np.ones(t.size, dtype=complex)
                        if f["slot"] >= 0:
                            fac = fac * slotv[f["slot"]]
                        rank = 0
                        for tt_ in range(5 + nw):
                            if (dm >> tt_) & 1:
                                on = ((tid >> tt_) & 1) == 1
                                fac = np.where(on, fac * slotv[f["dslot"] + rank], fac)
                                rank += 1
                    elif not (w0 >> 8) & 1:
                        fac = np.full(t.size, f["c"][0] + 1j * f["c"][1])
                        pb = (w0 >> 10) & 0xF
                        if pb:
                            sel &= ((tid >> (pb - 1)) & 1) == 1
                    else:
                        run = f["run"]
                        u = stat[f["row"] * nthreads + tid].copy()
                        if (w0 >> 9) & 1:
                            u += cst[run]
                        lr = ((w0 >> 14) & 0x1F) - 1
                        if lr >= 0:
                            u += lin[run * 16 + lr]
                        for tt_ in range(5 + nw):
                            if (dm >> tt_) & 1:
                                u += ((tid >> tt_) & 1) * lin[run * 16 + ttb[tt_]]
                        u &= MASK32
                        fac = np.exp(2j * np.pi * (u / 2.0 ** 32))
                    t[sel] *= fac[sel]
                if op == T2_DIAG:
                    continue
            # gates
            if ins["cls"] == C_REG:
                bit = reg[ins["idx"]]
            else:
                assert fmt == 1 and ins["cls"] == C_LANE and ins["idx"] < 5
                bit = lane[ins["idx"]]
            cond = None
            if ins["ccls"] == C_GLOBAL:
                if not ((base >> ins["cidx"]) & 1):
                    continue
            elif ins["ccls"] == C_REG:
                cond = ((loc >> reg[ins["cidx"]]) & 1) == 1
            elif ins["ccls"] == C_THREAD:
                cond = ((loc >> ttb[ins["cidx"]]) & 1) == 1
            if op in (T2_H, T2_HPH, T2_HG):  # T2_HG runs as H when the pass reads its state
                u = np.array([[1, 1], [1, -1]], dtype=complex)
            elif op == T2_ROT:  # shears a += t b, b += s a, a += t b (tileprog.h)
                tt, ss = (float(np.float32(v)) for v in t2["mats"][ins["aux"]][:2])
                sh_a = np.array([[1, tt], [0, 1]], dtype=complex)
                sh_b = np.array([[1, 0], [ss, 1]], dtype=complex)
                u = sh_a @ sh_b @ sh_a
            elif op == T2_X:
                u = np.array([[0, 1], [1, 0]], dtype=complex)
            else:
                u = mat_of(t2["mats"][ins["aux"]])
            apply_pairs(t, bit, u, cond)
        state[idx] = t


def run_general(state, gates):
    """A gate of the general set (physical qubits) by its definition: MCU
    acts where every control bit is 1; U2Q on the four amplitudes ordered by
    k = bit_a + 2 bit_b; MEASURE picks the smallest i with C_i > u C_last for
    C = (p0, p0 + p1), zeroes the other half and rescales the kept one.
    Returns the measurement outcome, or None."""
    x = np.arange(state.size)
    g0 = gates[0]
    if g0["kind"] == 11:  # MCU
        cm, t = int(g0["num"]), g0["target"]
        u = mat_of(g0["p"])
        apply_pairs(state, t, u, (x & cm) == cm)
        return None
    if g0["kind"] == 12:  # U2Q
        a, b = g0["target"], g0["control"]
        m4 = np.array([[complex(g["p"][2 * k], g["p"][2 * k + 1]) for k in range(4)] for g in gates])
        base = x[((x >> a) & 1 == 0) & ((x >> b) & 1 == 0)]
        idx = [base, base | (1 << a), base | (1 << b), base | (1 << a) | (1 << b)]
        v = np.stack([state[i] for i in idx])
        w = m4 @ v
        for k in range(4):
            state[idx[k]] = w[k]
        return None
    t, uval = g0["target"], g0["p"][0]
    bit = (x >> t) & 1
    q = np.abs(state) ** 2
    p0, p1 = float(np.sum(q[bit == 0])), float(np.sum(q[bit == 1]))
    out = 0 if p0 > uval * (p0 + p1) else 1
    keep = p0 if out == 0 else p1
    state[bit != out] = 0
    state[bit == out] /= np.sqrt(keep)
    return out


def remap(state, pairs):
    """Exchange the physical bit pairs of every index (a remap pass)."""
    x = np.arange(state.size)
    y = x.copy()
    for a, b in pairs:
        differ = ((x >> a) & 1) != ((x >> b) & 1)
        y = np.where(differ, y ^ ((1 << a) | (1 << b)), y)
    out = np.empty_like(state)
    out[y] = state
    return out


def product_state(n, basis, hq):
    """H^{hq}|basis> (H on the physical qubits of the mask hq)."""
    x = np.arange(1 << n)
    par = np.array([bin(int(i) & basis & hq).count("1") & 1 for i in x])
    v = 2.0 ** (-0.5 * bin(hq).count("1"))
    return np.where(((x ^ basis) & ~hq) == 0, np.where(par == 1, -v, v), 0.0).astype(complex)


def group_bases(n, p, group, b, tpb_log):
    """Physical tile bases of pass `p` inside block `b` of an L2 block group:
    the tile index's low bits run over the pass's global qubits inside the
    block, the block index over the qubits outside it."""
    allm = (1 << n) - 1
    inner = p["gmask"] & group["bmask"] & allm
    outer = p["gmask"] & ~group["bmask"] & allm
    return [pdep(t, inner) | pdep(b, outer) for t in range(1 << tpb_log)]


def run_plan(n, plan, use_gen=True, basis=0, hq=0, l2_groups=False):
    """Run the exported plan from the product state H^{hq}|basis> (default
    |0...0>).  With `use_gen` the first pass runs its generated-state variant
    (`t2gen`, as the library does from a recorded state) when it has one;
    otherwise every pass reads its state.  With `l2_groups` the passes of
    each exported L2 block group run (block, pass) segment by segment in the
    group's claim order."""
    state = product_state(n, basis, hq)
    first = True
    groups = {g["first"]: g for g in plan.get("l2_groups", [])} if l2_groups else {}
    skip = set()
    for i, p in enumerate(plan["passes"]):
        if i in skip:
            continue
        if i in groups:
            g = groups[i]
            if p.get("remap_before"):
                state = remap(state, p["remap_before"])
            tpb_log = g["l"] - p["k"]
            for s in g["segs"]:
                b, j = s >> 3, s & 7
                pj = plan["passes"][i + j]
                bases = group_bases(n, pj, g, b, tpb_log)
                if j == 0 and first and use_gen and "t2gen" in pj:
                    run_t2_pass(state, pj, pj["t2gen"], gen_basis=basis, gen_h=hq, bases=bases)
                else:
                    run_t2_pass(state, pj, bases=bases)
            skip.update(range(i + 1, i + g["count"]))
            first = False
            continue
        if p.get("general"):
            run_general(state, p["general"])
            first = False
            continue
        if p.get("remap_before"):
            state = remap(state, p["remap_before"])
        if not p["ops"]:
            continue
        if p["kernel"] in ("t2", "t3"):
            if first and use_gen and "t2gen" in p:
                run_t2_pass(state, p, p["t2gen"], gen_basis=basis, gen_h=hq)
            else:
                run_t2_pass(state, p)
        else:
            run_generic_pass(state, p)
        first = False
    # back to logical order
    phys = plan["phys"]
    x = np.arange(1 << n)
    y = np.zeros_like(x)
    for q in range(n):
        y |= ((x >> q) & 1) << phys[q]
    return state[y]
