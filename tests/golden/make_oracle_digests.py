"""Writes tests/golden/oracle_digests.txt: SHA-256 digests of the oracle's
frequencies and bitstreams on fixed seeded latents. Calls only oracle/ and
the input generator. Re-run only when the coder's definition changes, and
name the reason in the commit."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2509_18815_gb300 import synth  # noqa: E402

CASES = [
    # name, (C, H, W, K, seed, sigma_max, escape_stress), S
    ("latent_192x16x16_k3", (192, 16, 16, 3, 1001, 16.0, 0.0), 32),
    ("latent_8x16x16_k4_esc", (8, 16, 16, 4, 7, 16.0, 0.01), 64),
    ("latent_8x8x8_k3_s64max", (8, 8, 8, 3, 8, 64.0, 0.0), 96),
]


def digests():
    out = []
    for name, (C, H, W, K, seed, smax, esc), S in CASES:
        lat = synth.make_latent(C, H, W, K, seed, sigma_max=smax, escape_stress=esc)
        sf = oracle.freqs(lat.params, lat.symbols)
        words, offsets = oracle.encode(lat.params, lat.symbols, S)
        h_sf = hashlib.sha256(sf.tobytes()).hexdigest()
        h_w = hashlib.sha256(words.tobytes() + offsets.tobytes()).hexdigest()
        out.append((name, S, h_sf, h_w, int(words.size)))
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_digests.txt")
    with open(path, "w") as f:
        f.write("# written by tests/golden/make_oracle_digests.py (oracle only)\n")
        f.write("# name S sha256(freqs) sha256(words+offsets) n_words\n")
        for row in digests():
            f.write(" ".join(str(x) for x in row) + "\n")
    print(open(path).read())
