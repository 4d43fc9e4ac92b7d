"""Minimal Python reader of the program text format (test helper).

Reads only what the semantic checks need: the autoregressive output list,
the chain normalisation tables and the raw-channel columns of T.  Table
values are computed by the oracle's own C reader/evaluator.
"""


def read(path):
    toks = open(path).read().split()
    pos = 0

    def tok():
        nonlocal pos
        pos += 1
        return toks[pos - 1]

    def expect(w):
        t = tok()
        assert t == w, (w, t)

    expect("TSIMPROG"); tok()
    expect("mode"); mode = tok()
    hdr = {}
    for k in ("nx", "words", "nf", "nr", "nmeas", "ndet", "nobs"):
        expect(k)
        hdr[k] = int(tok())
    W = hdr["words"]
    words = lambda: [int(tok(), 16) for _ in range(W)]  # noqa: E731
    expect("outputs")
    outs = []
    for _ in range(int(tok())):
        t = tok()
        if t == "D":
            outs.append(("D", words(), int(tok())))
        else:
            outs.append(("R", int(tok()), int(tok()), int(tok())))
    expect("chains")
    chains = []
    for _ in range(int(tok())):
        expect("C")
        chains.append(int(tok()))
    expect("channels")
    channels = []
    for _ in range(int(tok())):
        expect("K")
        k = int(tok())
        thr = [int(tok()) for _ in range(k - 1)]
        sigs = []
        for _ in range(k):
            expect("S")
            sigs.append(words())
        channels.append((thr, sigs))
    expect("noise")
    noise_mode, ngroups = int(tok()), int(tok())
    groups = []
    for _ in range(ngroups):
        expect("G")
        q, m = int(tok()), int(tok())
        groups.append((q, [int(tok()) for _ in range(m)]))
    expect("tables")
    tables = []
    table_float = []
    for _ in range(int(tok())):
        expect("T")
        terms = []
        nt, fl = int(tok()), int(tok())
        for _ in range(nt):
            expect("t")
            s0, j0, m = int(tok()), int(tok()), int(tok())
            if fl:
                tok()  # the term's arbitrary phase (floating-point tables)
            facs = []
            for _ in range(m):
                expect("f")
                f = (int(tok()), int(tok()), int(tok()), words(), words())
                if f[0] == 4:
                    tok()  # the factor's arbitrary angle
                facs.append(f)
            terms.append((s0, j0, facs))
        tables.append(terms)
        table_float.append(fl)
    maps = {}
    for name in ("detmap", "obsmap"):
        expect(name)
        lst = []
        for _ in range(int(tok())):
            expect("M")
            lst.append([int(tok()) for _ in range(int(tok()))])
        maps[name] = lst
    expect("meta")
    meta = {}
    for _ in range(3):
        k = tok()
        meta[k] = int(tok())
    expect("raw")
    nraw, _ = int(tok()), int(tok())
    raw = []
    for _ in range(nraw):
        expect("Q")
        nb = int(tok())
        probs = [float(tok()) for _ in range(1 << nb)]
        cols = []
        for _ in range(nb):
            expect("B")
            cols.append(words())
        raw.append((nb, probs, cols))
    expect("end")
    return dict(mode=mode, outputs=outs, chains=chains, channels=channels, tables=tables, table_float=table_float,
                noise_mode=noise_mode, groups=groups,
                raw=raw, meta=meta, **hdr, **maps)


def x_of_raw(prog, e_bits):
    """X = T e in the program's X layout, from the raw columns (Eq. detector_sampling)."""
    x = [0] * prog["words"]
    b = 0
    for nb, _, cols in prog["raw"]:
        for i in range(nb):
            if e_bits[b]:
                for w in range(prog["words"]):
                    x[w] ^= cols[i][w]
            b += 1
    return x


def parity(mask, x):
    v = 0
    for m, w in zip(mask, x):
        v ^= m & w
    return bin(v).count("1") & 1
