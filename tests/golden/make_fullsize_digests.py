"""Writes tests/golden/fullsize_digests.json: SHA-256 digests of the CPU
reference's ciphertext words for the full-size cases of fullsize_cases.py.

Calls only the CPU reference (oracle/) and the seeded input module. Usage:
    python tests/golden/make_fullsize_digests.py [case ...] [--threads N]
With no case names every case is (re)computed; existing entries of other cases
are kept. The reference's threads only split loops with disjoint outputs, so
the digests do not depend on the thread count.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import oracle as O  # noqa: E402
import fullsize_cases as FC  # noqa: E402

OUT = os.path.join(HERE, "fullsize_digests.json")


def entry(ct):
    return dict(ncomp=ct.ncomp, level=ct.level, t_exp=ct.t_exp, sha256=FC.digest(ct.words()))


def context(params):
    o = O.Oracle(**params)
    o.keygen(o.rotate_sum_elements())
    return o


def run_ops(case):
    o = context(case["params"])
    va, vb = FC.ops_inputs(case, o.slots, o.t)
    a = o.encrypt(o.encode(va), 1)
    b = o.encrypt(o.encode(vb), 2)
    res = {"enc_a": a, "enc_b": b}
    res["tensor"] = o.tensor(a, b)
    res["relin"] = o.relin(res["tensor"])
    res["mul"] = o.mul(a, b)
    res["modswitch_1"] = o.modswitch(a, 1)
    res["modswitch_3"] = o.modswitch(a, 3)
    res["rotate_5"] = o.rotate(a, 5)
    res["rotate_m1"] = o.rotate(a, 2 * o.N - 1)
    res["rotate_sum"] = o.rotate_sum(res["mul"])
    for i, d in enumerate(o.reduce(a)):
        res["digit_%d" % i] = d
    assert list(res) == FC.OPS_RESULTS
    return {k: entry(v) for k, v in res.items()}


def run_query(case):
    o = context(case["params"])
    cols = FC.query_inputs(case, o.slots, o.t)
    enc = {k: [o.encrypt(o.encode(row), FC.NONCE[k] + i) for i, row in enumerate(v)]
           for k, v in cols.items() if not (case["square"] and k == "b")}
    if case["square"]:
        enc["b"] = enc["a"]
    res = o.query(enc["a"], enc["b"], enc["c1"], enc["c2"])
    out = {"result": entry(res), "noise_budget": o.noise_budget(res)}
    out["inputs"] = {"%s_%d" % (k, i): entry(c) for k, v in enc.items() for i, c in enumerate(v)}
    return out


def main(argv):
    names = [a for a in argv if not a.startswith("--")]
    if "--threads" in argv:
        O.set_threads(int(argv[argv.index("--threads") + 1]))
        names = [a for a in names if a != argv[argv.index("--threads") + 1]]
    names = names or list(FC.CASES)
    db = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        case = FC.CASES[name]
        t0 = time.time()
        res = run_ops(case) if case["kind"] == "ops" else run_query(case)
        db[name] = dict(results=res, seconds=round(time.time() - t0, 1), threads=O.threads())
        json.dump(db, open(OUT, "w"), indent=1, sort_keys=True)
        print("%s: %.1f s on %d threads" % (name, time.time() - t0, O.threads()), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
