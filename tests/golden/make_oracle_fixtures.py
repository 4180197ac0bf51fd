"""Writes oracle_fixtures.json: the first draws of a few streams of every
generator, computed by the CPU oracle alone (nothing else is imported).  The
fixture freezes the oracle: tests/test_golden.py checks that the oracle still
gives these values, and the GPU tests check the library against them.

Run from the repository root:  python tests/golden/make_oracle_fixtures.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402

N = 16          # draws per stream
STREAMS = 4     # streams per case
SEED = 0x5EED5EED5EED5EED
KEY_SEED = 0xC0FFEE


def cases():
    out = {}
    # MRG32k3a: streams 2^127 apart from the all-12345 state and from the expanded seed;
    # substreams 2^76 apart
    for name, seed_state, e in (("mrg32k3a_12345_streams", [12345] * 6, 127),
                                ("mrg32k3a_12345_substreams", [12345] * 6, 76),
                                ("mrg32k3a_seed_streams", [int(x) for x in O.seed_expand(SEED)], 127)):
        starts = O.mrg_stream_starts(seed_state, e, 0, STREAMS)
        vals, _ = O.mrg_bulk(starts, N)
        out[name] = {"seed_state": seed_state, "spacing_log2": e, "u32": vals.tolist(),
                     "f64": O.mrg_bulk(starts, N, O.OUT_F64)[0].tolist()}
    # Philox4x32-10: counter split (key = seed) and key per stream
    key = (KEY_SEED & 0xFFFFFFFF, KEY_SEED >> 32)
    out["philox4x32_10"] = {"seed": KEY_SEED,
                            "u32": O.philox_bulk(key, 0, [0] * STREAMS, N)[0].tolist()}
    out["philox4x32_10_keyed"] = {"seed": KEY_SEED,
                                  "u32": [O.philox_keyed_generate(KEY_SEED, s, 0, N).tolist()
                                          for s in range(STREAMS)]}
    out["threefry4x32_20"] = {"seed": KEY_SEED, "u32": O.threefry_bulk(KEY_SEED, 0, [0] * STREAMS, N)[0].tolist()}
    out["threefry4x64_20"] = {"seed": KEY_SEED, "u32": O.threefry64_bulk(KEY_SEED, 0, [0] * STREAMS, N)[0].tolist()}
    # TinyMT32: one parameter set found from the seed, its first streams (2^64 apart)
    prm = [int(x) for x in O.tinymt32_find_params(SEED, 1)[0]]
    starts = O.tinymt32_stream_starts(SEED & 0xFFFFFFFF, prm, 256, STREAMS)
    out["tinymt32"] = {"seed": SEED, "params": prm,
                       "u32": O.tinymt32_bulk(starts, prm, 256, N)[0].tolist()}
    return out


def main():
    path = os.path.join(HERE, "oracle_fixtures.json")
    c = cases()
    lines = [f'"{name}": ' + json.dumps(c[name], sort_keys=True) for name in sorted(c)]
    with open(path, "w") as f:
        f.write(f'{{"draws_per_stream": {N}, "streams": {STREAMS}, "cases": {{\n')
        f.write(",\n".join(lines))
        f.write("\n}}\n")
    print(path)


if __name__ == "__main__":
    main()
