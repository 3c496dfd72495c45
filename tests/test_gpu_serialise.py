"""The exchange format (pdq_cts_export/import, pdq_sk_export/import): bytes
written by the library equal the oracle's coefficient-form ciphertexts and
secret, bytes written from the oracle import and decrypt, and malformed
input is refused."""
import ctypes
import struct

import numpy as np
import pytest

from tests.gpu_common import Setup, library, to_np

pytestmark = pytest.mark.gpu

HDR = struct.Struct("<6I2Q24x")          # magic, version, N, limbs, level, count, t, q0
MAGIC_CTS, MAGIC_SK = 0x43514450, 0x53514450


@pytest.fixture(scope="module")
def st():
    return Setup("tiny2")


def _header(par, magic, count):
    return HDR.pack(magic, 1, par.N, par.L, par.L, count, par.t, par.q[0])


def test_export_is_the_oracle_ciphertext(st):
    data = st.ctx.cts_export(st.v_cts)
    J = st.oplan.J
    assert data[:HDR.size] == _header(st.par, MAGIC_CTS, J)
    got = np.frombuffer(data[HDR.size:], dtype="<u8").reshape(J, 2, st.par.L, st.par.N)
    want = np.asarray(st.o_v_cts, dtype=np.uint64).reshape(J, 2, st.par.L, st.par.N)
    assert np.array_equal(got, want)


def test_oracle_bytes_import_and_decrypt(st):
    J = st.oplan.J
    want = np.asarray(st.o_v_cts, dtype=np.uint64).reshape(J, 2, st.par.L, st.par.N)
    data = _header(st.par, MAGIC_CTS, J) + want.astype("<u8").tobytes()
    ct = st.ctx.cts_import(data)
    assert np.array_equal(to_np(ct), to_np(st.v_cts.view(J, 2, st.par.L, st.par.N)))
    slots = st.ctx.decrypt(st.sk, ct).cpu().numpy().astype(np.int64)
    assert np.array_equal(slots, st.v_slots.astype(np.int64))
    assert st.ctx.cts_export(ct) == data


def test_secret_round_trip(st):
    data = st.ctx.sk_export(st.sk)
    assert data[:HDR.size] == _header(st.par, MAGIC_SK, 1)
    s = np.frombuffer(data[HDR.size:], dtype=np.int8)
    assert np.array_equal(s, np.asarray(st.q.sk, dtype=np.int8))
    back = st.ctx.sk_import(data)
    assert np.array_equal(to_np(back), to_np(st.sk))


def test_malformed_input_is_refused(st):
    pdq = library()
    J = st.oplan.J
    good = st.ctx.cts_export(st.v_cts)
    bad_magic = struct.pack("<I", 0x12345678) + good[4:]
    with pytest.raises(pdq.PdqError):
        st.ctx.cts_import(bad_magic)
    with pytest.raises(pdq.PdqError):
        st.ctx.cts_import(good[:-8])                    # truncated payload
    hdr = bytearray(good[:HDR.size])
    hdr[8:12] = struct.pack("<I", st.par.N * 2)         # another ring
    with pytest.raises(pdq.PdqError):
        st.ctx.cts_import(bytes(hdr) + good[HDR.size:])
    big = np.frombuffer(good[HDR.size:], dtype="<u8").copy()
    big[0] = st.par.q[0]                                # not canonical
    with pytest.raises(pdq.PdqError):
        st.ctx.cts_import(good[:HDR.size] + big.tobytes())
    # room for fewer ciphertexts than the header holds
    lib = pdq.load()
    out = st.ctx._u64(st.ctx.ct_elems)
    cnt = ctypes.c_uint32()
    rc = lib.pdq_cts_import(st.ctx.h, good, len(good), out.data_ptr(), 0, ctypes.byref(cnt), None)
    assert rc == 2 and cnt.value == J                   # PDQ_E_NOMEM
    # a secret that is not ternary
    sk = bytearray(st.ctx.sk_export(st.sk))
    sk[HDR.size] = 2
    with pytest.raises(pdq.PdqError):
        st.ctx.sk_import(bytes(sk))


KHDR = struct.Struct("<6I2QI20x")        # ... + the digit count in the reserved bytes
MAGIC_KEYS = 0x4B514450


def _oracle_key_bytes(st, order):
    par = st.par
    body = np.stack([np.asarray(st.o_keys[k], dtype=np.uint64) for k in order])
    return (KHDR.pack(MAGIC_KEYS, 1, par.N, par.L + par.K, par.L, len(order), par.t, par.q[0],
                      len(par.digits))
            + np.asarray(order, dtype="<u8").tobytes() + body.astype("<u8").tobytes())


def test_rotation_key_export_is_the_oracle_keys(st):
    data = st.ctx.rotkeys_export(st.keys, st.galois)
    assert data == _oracle_key_bytes(st, st.galois)


def test_oracle_rotation_keys_import_and_answer_bit_exact(st):
    """Keys made by the oracle (another implementation of the key equation)
    enter the library, in an order other than the plan's, and the Answer
    with them is the oracle's Answer bit for bit."""
    from oracle import pdq as opdq
    from tests.gpu_common import coeff
    order = list(reversed(st.galois))
    keys, gal = st.ctx.rotkeys_import(_oracle_key_bytes(st, order))
    assert gal == order
    out = st.ctx.answer(st.plan, st.v_cts, st.db, keys, gal, st.consts)
    got = coeff(st.ctx, out, st.par.L)
    want = opdq.answer(st.par, st.o_v_cts, st.q.db, st.o_keys, st.oplan)
    for c, w in enumerate(want):
        assert np.array_equal(got[c], w)
    # and the imported keys export to the same bytes
    assert st.ctx.rotkeys_export(keys, gal) == _oracle_key_bytes(st, order)


def test_malformed_rotation_keys_are_refused(st):
    pdq = library()
    good = _oracle_key_bytes(st, st.galois[:2])
    par = st.par

    def refused(data, code=pdq.PDQ_E_PARAM):
        with pytest.raises(pdq.PdqError) as e:
            st.ctx.rotkeys_import(data)
        assert e.value.code == code

    refused(good[:-8])                                            # truncated
    refused(struct.pack("<I", MAGIC_CTS) + good[4:])              # a ciphertext header
    hdr = bytearray(good[:KHDR.size])
    hdr[40:44] = struct.pack("<I", len(par.digits) + 1)           # another digit count
    refused(bytes(hdr) + good[KHDR.size:])
    hdr = bytearray(good[:KHDR.size])
    hdr[12:16] = struct.pack("<I", par.L)                         # limbs without the special primes
    refused(bytes(hdr) + good[KHDR.size:])
    gal = bytearray(good)
    gal[KHDR.size:KHDR.size + 8] = struct.pack("<Q", 2)           # even Galois element
    refused(bytes(gal))
    gal[KHDR.size:KHDR.size + 8] = good[KHDR.size + 8:KHDR.size + 16]   # repeated element
    refused(bytes(gal))
    body = np.frombuffer(good, dtype="<u8", offset=KHDR.size + 16).copy()
    body[par.N] = par.ext[1]                                      # limb 1 not canonical
    refused(good[:KHDR.size + 16] + body.tobytes())
    lib = pdq.load()
    out = st.ctx._u64(2 * st.ctx.key_elems)
    g = np.zeros(2, dtype=np.uint64)
    cnt = ctypes.c_uint32()
    rc = lib.pdq_rotkeys_import(st.ctx.h, good, len(good), out.data_ptr(), g.ctypes.data, 1,
                                ctypes.byref(cnt), None)
    assert rc == pdq.PDQ_E_NOMEM and cnt.value == 2
