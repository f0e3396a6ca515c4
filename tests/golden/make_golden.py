"""Write the stored oracle outputs used by the GPU parity tests.

Every value written here comes from ``oracle/`` (FP64 CPU) run on the seeded
inputs of ``gen/``; nothing comes from the CUDA path.  Each file records the
workload, its seed and the SHA-256 prefix of the generated float32 data, so a
test can refuse to compare against data that drifted.

    python tests/golden/make_golden.py cfg1 cfg2 cfg4 cfg5 cfg3 long_n rows [--threads N]

`rows` (run after the orders) writes oracle_rows.json: first-step scores of
sampled variables and adjacency rows along the stored orders, which bench.py
reads to state each GPU form's error against the oracle.

cfg3 (d=1000, n=10000) is ~1e5 core-seconds of FP64 libm work.
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gen      # noqa: E402
import oracle   # noqa: E402

def write_order(name, order, header_lines):
    path = os.path.join(HERE, f"{name}_order.txt")
    with open(path + ".tmp", "w") as f:
        for h in header_lines:
            f.write(f"# {h}\n")
        f.write(" ".join(str(int(v)) for v in order) + "\n")
    os.replace(path + ".tmp", path)
    print("wrote", path, flush=True)


def header(workload, digest, seconds, threads):
    return [
        "DirectLiNGAM causal order from the FP64 oracle (oracle.causal_order, memoised mode,",
        "bitwise identical to the literal Algorithm 1 loop).",
        f"workload: {workload}",
        f"data-sha256-16: {digest}",
        f"oracle wall seconds: {seconds:.1f} on {threads} threads",
        "written by tests/golden/make_golden.py",
    ]


def run_cfg(k, threads):
    ds = getattr(gen, f"cfg{k}")()
    t = time.time()
    order = oracle.causal_order(ds.X, threads=threads)
    write_order(f"cfg{k}", order,
                header(f"cfg{k} d={ds.d} n={ds.n} seed={gen.SEEDS[k]}", ds.digest(),
                       time.time() - t, threads))


def run_long_n(threads):
    ds = gen.long_n()
    t = time.time()
    order = oracle.causal_order(ds.X, threads=threads)
    write_order("long_n", order,
                header(f"long_n d={ds.d} n={ds.n} seed={gen.SEEDS[6]}", ds.digest(),
                       time.time() - t, threads))


def run_cfg4(threads):
    vd = gen.cfg4()
    t = time.time()
    M, E = oracle.var_fit(vd.Xt, 1)
    order = oracle.causal_order(E, threads=threads)
    write_order("cfg4", order,
                header(f"cfg4 VarLiNGAM innovations d={vd.Xt.shape[1]} T={vd.Xt.shape[0]} lag=1 "
                       f"seed={gen.SEEDS[4]}", vd.digest(), time.time() - t, threads))


def _read_cfg5(path):
    """Instances already stored: {index: line} (the file is rewritten after each one)."""
    done = {}
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                done[int(line.split()[0])] = line if line.endswith("\n") else line + "\n"
    return done


def run_cfg5(threads):
    """Oracle orders of all 192 batch instances, cheapest first.

    The file is rewritten (sorted by instance index) after every instance, so
    an interrupted run keeps what it finished and a rerun skips it."""
    import hashlib
    insts = gen.cfg5()
    path = os.path.join(HERE, "cfg5_orders.txt")
    done = _read_cfg5(path)
    todo = [k for k in range(len(insts)) if k not in done]
    n_of = [len(i.rows) if i.rows is not None else i.X.shape[0] for i in insts]
    todo.sort(key=lambda k: (gen.residual_samples(insts[k].X.shape[1], n_of[k]), k))
    for k in todo:
        X = insts[k].data()
        dig = hashlib.sha256(np.ascontiguousarray(X).tobytes()).hexdigest()[:16]
        t = time.time()
        order = oracle.causal_order(X, threads=threads)
        print(f"cfg5[{k}] {insts[k].name} d={X.shape[1]} n={X.shape[0]} "
              f"{time.time() - t:.1f}s", flush=True)
        done[k] = f"{k} {insts[k].name} {dig} : " + " ".join(str(int(v)) for v in order) + "\n"
        with open(path + ".tmp", "w") as f:
            f.write("# DirectLiNGAM causal orders from the FP64 oracle for the cfg5 instances.\n")
            f.write(f"# workload: cfg5 seed={gen.SEEDS[5]}; one line per instance:\n")
            f.write("# <instance index> <name> <data-sha256-16> : <order>\n")
            f.write("# written by tests/golden/make_golden.py\n")
            for j in sorted(done):
                f.write(done[j])
        os.replace(path + ".tmp", path)
    print("wrote", path, f"({len(done)} instances)", flush=True)


ROW_SAMPLES = {"cfg1": None, "cfg2": None, "cfg3": [0, 1, 137, 500, 998, 999],
               "cfg4": [0, 5, 200, 486], "long_n": [0, 3, 41, 77, 99]}
B_SAMPLES = {"cfg1": None, "cfg2": [0, 17, 50, 99], "cfg3": [0, 137, 500, 999],
             "cfg4": [0, 5, 200, 486], "long_n": [0, 41, 99]}


def run_rows(threads):
    """Sampled first-step scores and adjacency rows of the FP64 oracle per
    workload (None = every variable), along the stored oracle orders."""
    import json
    from gpu_util_golden import read_order
    out = {}
    for name in ROW_SAMPLES:
        if name == "cfg4":
            vd = gen.cfg4()
            M, X = oracle.var_fit(vd.Xt, 1)
            digest = vd.digest()
        else:
            ds = gen.long_n() if name == "long_n" else getattr(gen, name)()
            X, digest = ds.X.astype(np.float64), ds.digest()
        order, gdig = read_order(os.path.join(HERE, f"{name}_order.txt"))
        if order is None or gdig != digest:
            print(f"rows: {name} has no stored order for this data; skipped", flush=True)
            continue
        t = time.time()
        d = X.shape[1]
        sv = ROW_SAMPLES[name]
        if sv is None:
            sv = list(range(d))
            m = oracle.search_step(X, threads=threads)["k_list"]
        else:
            m = oracle.row_scores(X, sv, threads=threads)
        bv = B_SAMPLES[name] or list(range(d))
        B = oracle.adjacency_rows(X, order, bv)
        out[name] = {"data_sha256_16": digest, "step0_vars": [int(v) for v in sv],
                     "step0_M": [float(v) for v in m], "B_vars": [int(v) for v in bv],
                     "B_rows": [[float(v) for v in row] for row in B]}
        print(f"rows: {name} {time.time() - t:.1f}s", flush=True)
    path = os.path.join(HERE, "oracle_rows.json")
    with open(path + ".tmp", "w") as f:
        f.write(json.dumps({"written_by": "tests/golden/make_golden.py rows (oracle/ only)",
                            "what": "FP64 oracle: first-step k_list of sampled variables "
                                    "(Algorithm 1) and adjacency rows B[v] along the stored "
                                    "oracle order (least squares on the predecessors)",
                            "workloads": out}, indent=1))
    os.replace(path + ".tmp", path)
    print("wrote", path, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", nargs="+")
    ap.add_argument("--threads", type=int, default=oracle.default_threads())
    a = ap.parse_args()
    for w in a.which:
        if w in ("cfg1", "cfg2", "cfg3"):
            run_cfg(int(w[-1]), a.threads)
        elif w == "cfg4":
            run_cfg4(a.threads)
        elif w == "cfg5":
            run_cfg5(a.threads)
        elif w == "long_n":
            run_long_n(a.threads)
        elif w == "rows":
            run_rows(a.threads)
        else:
            raise SystemExit(f"unknown workload {w}")


if __name__ == "__main__":
    main()
