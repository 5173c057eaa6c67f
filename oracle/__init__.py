"""CPU reference oracle for the encrypted quadratic-gradient NAG iteration.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product package.  It shares no code
with the CUDA path.

* ``he_oracle.c``  -- RNS-CKKS primitives in plain C (128-bit products, ``%``).
* ``ckks.py``      -- ciphertext objects and scale bookkeeping over those primitives.
* ``qgnag.py``     -- client precompute and the encrypted QG-NAG iteration (Sec. 3-4).
* ``plain.py``     -- the same algorithm in FP64 on plaintext (Algorithm 1).
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "he_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libheoracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile he_oracle.c with gcc (no FP contraction, OpenMP over limbs)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(L):
    u64, i64, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                              ctypes.c_double, ctypes.c_void_p)
    sig = {
        "orc_is_prime": (i32, [u64]),
        "orc_gen_primes": (i32, [i32, i32, i32, i32, i32, vp]),
        "orc_find_psi": (u64, [u64, i32]),
        "orc_ntt_direct": (None, [i32, u64, u64, vp, vp]),
        "orc_polymul_schoolbook": (None, [i32, u64, vp, vp, vp]),
        "orc_rand_word": (u64, [u64, u64, u64]),
        "orc_splitmix64_next": (u64, [vp]),
        "orc_cdt_table": (i32, [dbl, vp, i32]),
        "orc_sample": (None, [u64, u64, i32, u64, dbl, i64, vp]),
        "orc_ctx_new": (vp, [i32, i32, i32, i32, i32, dbl]),
        "orc_ctx_new_bits": (vp, [i32, i32, vp, i32, dbl]),
        "orc_gen_primes_bits": (i32, [i32, i32, vp, i32, vp]),
        "orc_set_secret_weight": (i32, [vp, i32]),
        "orc_ctx_free": (None, [vp]),
        "orc_get_primes": (None, [vp, vp]),
        "orc_get_psi": (None, [vp, vp]),
        "orc_get_zeta_table": (None, [vp, vp, vp]),
        "orc_get_cdt": (i32, [vp, vp]),
        "orc_get_sk": (None, [vp, vp]),
        "orc_ntt": (None, [vp, i32, vp]),
        "orc_intt": (None, [vp, i32, vp]),
        "orc_polymul": (None, [vp, i32, vp, vp, vp]),
        "orc_embed_inv": (None, [vp, vp, vp, vp]),
        "orc_embed": (None, [vp, vp, vp, vp]),
        "orc_encode": (i32, [vp, vp, vp, i32, dbl, vp]),
        "orc_decode": (None, [vp, vp, dbl, vp, vp]),
        "orc_automorph": (None, [vp, i32, u64, vp, vp]),
        "orc_keygen": (i32, [vp, u64, vp, i32]),
        "orc_encrypt": (None, [vp, vp, i32, u64, vp]),
        "orc_decrypt": (None, [vp, vp, i32, vp]),
        "orc_decrypt3": (None, [vp, vp, i32, vp]),
        "orc_add": (None, [vp, i32, i32, vp, vp, vp, i32]),
        "orc_tensor": (None, [vp, i32, vp, vp, vp]),
        "orc_keyswitch": (i32, [vp, i32, u64, vp, vp]),
        "orc_relin": (i32, [vp, i32, vp, vp]),
        "orc_rotate_gal": (i32, [vp, i32, u64, vp, vp]),
        "orc_galois_elt": (u64, [vp, i64]),
        "orc_rotate": (i32, [vp, i32, i64, vp, vp]),
        "orc_rotsum_gal": (i32, [vp, i32, vp, i32, vp, vp]),
        "orc_rescale": (None, [vp, i32, i32, vp, vp]),
        "orc_moddrop": (None, [vp, i32, i32, i32, vp, vp]),
        "orc_cmul_int": (None, [vp, i32, i32, vp, i64, vp]),
        "orc_cadd_int": (None, [vp, i32, vp, i64, vp]),
        "orc_ptmul": (None, [vp, i32, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L
