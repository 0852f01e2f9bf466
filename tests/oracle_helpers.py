"""Test plumbing around the FP64 oracle: momentum sums, and copies of the
oracle compiled with one mistake planted in its source, so that a pin can be
shown to fail on the kind of mistake it is there to catch."""
import hashlib
import os
import subprocess

import numpy as np

import oracle

_VARIANT_DIR = os.path.join(oracle.OUT_DIR, "planted")


def momentum(pop, e):
    """Total momentum sum_x sum_a e_a f_a(x) of a [19, ...] population array."""
    flat = pop.reshape(19, -1).sum(axis=1)
    return e.T.astype(np.float64) @ flat


def planted(old: str, new: str):
    """The oracle compiled from its source with the single occurrence of
    ``old`` replaced by ``new``; returns the loaded library (for
    ``oracle.Oracle(..., lib=...)``)."""
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"planted mistake does not match the oracle source once: {old!r}"
    text = src.replace(old, new)
    tag = hashlib.sha1(text.encode()).hexdigest()[:16]
    os.makedirs(_VARIANT_DIR, exist_ok=True)
    so = os.path.join(_VARIANT_DIR, f"lbm_oracle_{tag}.so")
    if not os.path.exists(so):
        c = os.path.join(_VARIANT_DIR, f"lbm_oracle_{tag}.c")
        with open(c, "w") as fh:
            fh.write(text)
        tmp = so + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-D_DEFAULT_SOURCE",
                        "-I", oracle.HERE, "-o", tmp, c, "-lm"], check=True)
        os.replace(tmp, so)
    return oracle.load(so)
