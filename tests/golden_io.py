"""Reader for tests/golden/hand_examples.txt (no arithmetic of the method)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def hand_examples():
    out = []
    with open(os.path.join(GOLDEN, "hand_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, Fs, ms, ds, dins, mss = [p.split() for p in line.split("|")]
            name, Nt, Nd, Nm = head[0], int(head[1]), int(head[2]), int(head[3])
            arr = lambda xs, shp: np.array([float(x) for x in xs]).reshape(shp)
            out.append(dict(name=name, Nt=Nt, Nd=Nd, Nm=Nm,
                            Fcol=arr(Fs, (Nt, Nd, Nm)), m=arr(ms, (Nt, Nm)), d=arr(ds, (Nt, Nd)),
                            d_in=arr(dins, (Nt, Nd)), mstar=arr(mss, (Nt, Nm))))
    return out
