"""Hand-written compiled programs for oracle pins (test helper).

Formats the program text layout read by both the oracle and the product
(documented with ``tsim_program_save`` in include/tsim.h) from plain Python
lists, so that tests can state tiny programs whose marginals are known in
closed form.
"""


def hexw(words):
    return " ".join(f"{w & 0xFFFFFFFFFFFFFFFF:016x}" for w in words)


def program_text(*, mode="detectors", nx=1, nf=0, nr=0, nmeas=0, ndet=0, nobs=0,
                 outputs=(), chains=(), channels=(), tables=(), detmap=(), obsmap=(), groups=None):
    """outputs: ("D", mask_words, const) | ("R", xbit, chain, table)
    channels: (thresholds, [sig words per outcome])
    groups: None (one word per channel) or [(Q, [channel indices])] (geometric gaps)
    tables: [terms], term = (s0, j0, [(kind, alpha, beta, u_words, v_words)])"""
    W = max(1, (nx + 63) // 64)
    L = ["TSIMPROG 2", f"mode {mode}", f"nx {nx}", f"words {W}", f"nf {nf}", f"nr {nr}",
         f"nmeas {nmeas}", f"ndet {ndet}", f"nobs {nobs}", f"outputs {len(outputs)}"]
    for o in outputs:
        if o[0] == "D":
            L.append(f"D {hexw(o[1])} {o[2]}")
        else:
            L.append(f"R {o[1]} {o[2]} {o[3]}")
    L.append(f"chains {len(chains)}")
    for c in chains:
        L.append(f"C {c}")
    L.append(f"channels {len(channels)}")
    for thr, sigs in channels:
        L.append(f"K {len(sigs)} " + " ".join(str(t) for t in thr))
        for s in sigs:
            L.append(f"S {hexw(s)}")
    if groups is None:
        L.append("noise 0 0")
    else:
        L.append(f"noise 1 {len(groups)}")
        for Q, members in groups:
            L.append(f"G {Q} {len(members)} " + " ".join(str(c) for c in members))
    L.append(f"tables {len(tables)}")
    for terms in tables:
        L.append(f"T {len(terms)} 0")
        for s0, j0, facs in terms:
            L.append(f"t {s0} {j0} {len(facs)}")
            for kind, a, b, u, v in facs:
                L.append(f"f {kind} {a} {b} {hexw(u)} {hexw(v)}")
    L.append(f"detmap {len(detmap)}")
    for d in detmap:
        L.append(f"M {len(d)} " + " ".join(str(j) for j in d))
    L.append(f"obsmap {len(obsmap)}")
    for d in obsmap:
        L.append(f"M {len(d)} " + " ".join(str(j) for j in d))
    L.append("raw 0 0")
    L.append("end")
    return "\n".join(L) + "\n"
