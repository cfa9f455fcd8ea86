"""Write packed_f32_zero_fringe.json: for each distribution, a counter whose
packed-keying FP32 draw leaves step 2 (layer index >= L_max) with U = 0, so
that a GPU test checks a fringe draw whose first overhang attempt starts
at u_x = 0 (for the normal, one whose sign bit is set).  Runs
find_packed_zero.c against the oracle's Philox only (oracle/liborc.so),
on all host cores; it finds both counters within seconds."""
import json
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402

SEED = 0x0123456789ABCDEF
CHUNK = 1 << 26


def main():
    lib = oracle.build()
    exe = os.path.join(HERE, "_find_packed_zero")
    subprocess.run(["gcc", "-O2", os.path.join(HERE, "find_packed_zero.c"), lib, "-o", exe,
                    f"-Wl,-rpath,{os.path.dirname(lib)}"], check=True)
    out = {"seed": SEED, "note": "counters whose packed-keying FP32 first word has a layer "
           "index >= L_max and U = 0 (bits 9-31 zero), the normal's with its sign bit set, found "
           "with the oracle's Philox"}
    for name, dist in (("exp", oracle.EXP), ("normal", oracle.NORMAL)):
        L = oracle.tables(dist).L

        def run(c):
            r = subprocess.run([exe, str(SEED), str(L), str(int(dist == oracle.NORMAL)),
                                str(c * CHUNK), str(CHUNK)],
                               capture_output=True, text=True, check=True)
            return int(r.stdout.strip())

        found = -1
        with ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
            for base in range(0, 256, os.cpu_count()):
                hits = [g for g in ex.map(run, range(base, base + os.cpu_count())) if g >= 0]
                if hits:
                    found = min(hits)
                    break
        out[name] = found
        print(name, L, found, flush=True)
    os.remove(exe)
    with open(os.path.join(HERE, "packed_f32_zero_fringe.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
