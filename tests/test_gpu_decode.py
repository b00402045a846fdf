"""GPU parity of the decode path against the CPU oracle, through the C ABI.

Every case compares the GPU output byte for byte with the oracle's
sequential decode and checks the GPU FNV against the oracle FNV (integer
work: the bar is bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_2607_18541_gb300 import aclz, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    aclz.lib()  # raises if libaclz.so is missing: no fallback


# (mode, flags): the wave schedule, and the persistent schedule with each
# copy path
WAVES = (aclz.ACLZ_MODE_WAVES, 0)
PERSIST_STAGED = (aclz.ACLZ_MODE_PERSISTENT, aclz.ACLZ_FLAG_STAGED)
PERSIST_REGS = (aclz.ACLZ_MODE_PERSISTENT, aclz.ACLZ_FLAG_REGISTERS)
MODES = (WAVES, PERSIST_STAGED, PERSIST_REGS)


def gpu_decode(c, G=32, mode=WAVES, fnv=True, range_bytes=None, ctas_per_sm=0, phase_event=None,
               flatten=False):
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        if flatten:
            aclz.aclz_flatten(h, s)
        info = aclz.aclz_handle_info(h)
        if range_bytes:
            aclz.aclz_set_range_bytes(h, range_bytes, s)
        out = torch.empty(max(16, (info.total_len + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
        if phase_event is not None:
            aclz.aclz_decode_all_ev(h, out, phase_event, G=G, mode=mode[0], flags=mode[1],
                                    ctas_per_sm=ctas_per_sm, stream=s)
        else:
            aclz.aclz_decode_all(h, out, G=G, mode=mode[0], flags=mode[1], ctas_per_sm=ctas_per_sm, stream=s)
        assert aclz.aclz_device_status(h, s) == aclz.ACLZ_OK
        got = out[:info.total_len].cpu().numpy()
        f = aclz.aclz_fnv(out, info.total_len, stream=s) if fnv else None
        return got, f, h_info_dict(h)
    finally:
        aclz.aclz_free(h)


def h_info_dict(h):
    i = aclz.aclz_handle_info(h)
    return dict(n_waves=i.n_waves, n_deferred=i.n_deferred, n_tokens=i.n_tokens)


def check(c, G=32, modes=MODES):
    """Decode c in each mode; byte compare and FNV against the oracle."""
    exp = oracle.decode(c)
    fe = oracle.fnv_chunked(exp)
    for mode in modes:
        got, f, info = gpu_decode(c, G, mode)
        assert got.size == exp.size
        if not np.array_equal(got, exp):
            bad = np.nonzero(got != exp)[0]
            raise AssertionError(f"{bad.size} bytes differ, first at {bad[0]} (G={G}, mode={mode})")
        assert f == fe
    return info


# ------------------------------------------------------ workload configs

def test_markov_4mib_base_thresholds_64k_blocks_g32():
    """4 MiB order-2 Markov, 6/8/10/12, 64 KiB blocks, G = 32."""
    x = synth.markov2(4 << 20, seed=synth.SEED_MARKOV)
    c = oracle.encode(x, 1 << 16, oracle.PRESET_BASE)
    info = check(c, 32)
    assert info["n_waves"] >= 2
    assert np.array_equal(oracle.decode(c), x)


@pytest.mark.parametrize("G", [8, 16, 32])
@pytest.mark.parametrize("L", [32, 64, 256, 1024])
def test_copy_sweep_small(G, L):
    sw = synth.copy_sweep((8 << 20) + 12345, 1 << 14, L, seed=100 + L)
    check(oracle.pack_sweep(sw, tags=False), G)


@pytest.mark.parametrize("bs", [1 << 12, 1 << 15, 1 << 17])
def test_copy_sweep_block_sizes(bs):
    sw = synth.copy_sweep(6 << 20, bs, 128, seed=bs)
    check(oracle.pack_sweep(sw, tags=False), 32)


@pytest.mark.parametrize("preset", [0, 1, 2])
def test_fastq_presets(preset):
    x = synth.fastq(3 << 20, seed=77)
    mm = (oracle.PRESET_BASE, oracle.PRESET_TUNED, oracle.PRESET_PUSH)[preset]
    check(oracle.encode(x, 1 << 14, mm), 32)


def test_wordtext_and_product_encoder():
    x = synth.wordtext(3 << 20, seed=5, chunk_bytes=1 << 20)
    p = aclz.aclz_encode_params_default(aclz.ACLZ_PRESET_TUNED)
    p.block_size = 1 << 16
    c = aclz.aclz_encode(x, p)
    for mode in MODES:
        got, f, _ = gpu_decode(c, 16, mode)
        assert np.array_equal(got, x)
        assert f == oracle.fnv_chunked(x)


@pytest.mark.parametrize("range_bytes", [64, 4096, 1 << 20])
@pytest.mark.parametrize("mode", [PERSIST_STAGED, PERSIST_REGS])
def test_persistent_range_sizes(range_bytes, mode):
    """Ranges from 8 matches (more segments than lanes) to 4096 matches."""
    x = synth.markov2(2 << 20, seed=17)
    c = oracle.encode(x, 1 << 12, oracle.PRESET_BASE)
    sw = synth.copy_sweep(4 << 20, 1 << 13, 512, seed=18)
    c2 = oracle.pack_sweep(sw, tags=False)
    for cc, G in ((c, 32), (c2, 8), (c2, 32)):
        exp = oracle.decode(cc)
        got, f, _ = gpu_decode(cc, G, mode, range_bytes=range_bytes)
        assert np.array_equal(got, exp)
        assert f == oracle.fnv_chunked(exp)


# ------------------------------------------------------------ wave tags

@pytest.mark.parametrize("kind", ["markov", "sweep", "fastq"])
def test_gpu_tags_equal_oracle_minimal_tags(kind):
    if kind == "markov":
        c = oracle.encode(synth.markov2(2 << 20, seed=3), 1 << 12, oracle.PRESET_BASE)
    elif kind == "sweep":
        c = oracle.pack_sweep(synth.copy_sweep(4 << 20, 1 << 12, 48, seed=4))
    else:
        c = oracle.encode(synth.fastq(2 << 20, seed=5), 1 << 12, oracle.PRESET_BASE)
    want, nw = oracle.min_tags(c)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(oracle.strip_tags(c), s)  # GPU computes the tags
    try:
        got = aclz.aclz_tags(h)
        assert aclz.aclz_handle_info(h).n_waves == nw
    finally:
        aclz.aclz_free(h)
    assert np.array_equal(got, want)


def test_given_and_nonminimal_tags_decode_identically():
    x = synth.markov2(3 << 20, seed=8)
    c = oracle.encode(x, 1 << 13, oracle.PRESET_BASE)       # minimal tags present
    extra = np.random.default_rng(1).integers(0, 4, oracle.header(c).n_tokens).astype(np.uint32)
    c2 = oracle.retag(c, extra)                               # legal, non-minimal
    assert oracle.validate(c2) == 0
    for cc in (c, c2, oracle.strip_tags(c)):
        for mode in MODES:
            got, _, info = gpu_decode(cc, 32, mode)
            assert np.array_equal(got, x)


# ------------------------------------------------------------ edge cases

@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 4095, 70000])
def test_edge_sizes(n):
    x = synth.markov2(max(n, 1), seed=11)[:n]
    c = oracle.encode(x, 1 << 12, oracle.PRESET_BASE)
    if n == 0:
        s = torch.cuda.current_stream()
        h = aclz.aclz_upload(c, s)
        out = torch.empty(16, dtype=torch.uint8, device="cuda")
        aclz.aclz_decode_all(h, out, stream=s)
        assert aclz.aclz_device_status(h, s) == 0
        aclz.aclz_free(h)
        return
    check(c, 8)


def test_tiny_blocks_deep_waves_and_single_huge_block():
    x = synth.markov2(200_000, seed=12)
    check(oracle.encode(x, 64, (4, 4, 4, 4)), 32)          # 64-byte blocks, many waves
    check(oracle.encode(x, 1 << 24, oracle.PRESET_BASE), 16)  # one 16 MiB block
    z = np.zeros(300_000, dtype=np.uint8)                     # constant run: doubling chain
    check(oracle.encode(z, 1 << 12, oracle.PRESET_BASE, chain_depth=oracle.UNLIMITED_DEPTH), 32)
    r = np.frombuffer(np.random.default_rng(0).bytes(100_000), dtype=np.uint8)  # literal only
    check(oracle.encode(r, 1 << 12, oracle.PRESET_BASE), 32)


def test_misaligned_sources_and_in_block_chains():
    # matches at every alignment of src and dst mod 16, chains inside a block
    rng = np.random.default_rng(3)
    blk, ll, ml, sr, lits = [], [], [], [], bytearray()
    total, bs = 0, 1 << 12
    for b in range(64):
        pos, cnt = b * bs, 0
        end = pos + bs
        while pos < end:
            lit = int(rng.integers(0, 20))
            m = int(rng.integers(1, 80))
            if pos + lit + m <= end and pos + lit >= m:
                src = int(rng.integers(max(0, pos + lit - 3000), pos + lit - m + 1))
                ll.append(lit); ml.append(m); sr.append(src)
                lits += rng.bytes(lit)
                pos += lit + m
            else:
                ll.append(end - pos); ml.append(0); sr.append(0)
                lits += rng.bytes(end - pos)
                pos = end
            cnt += 1
        blk.append(cnt)
        total = end
    c = oracle.pack(total, bs, blk, ll, ml, sr, bytes(lits), tags=False)
    for G in (8, 16, 32):
        check(c, G)


def test_mixed_length_matches_long_on_average():
    # deferred matches of 1..400 bytes averaging well over three 16-byte
    # chunks, at every alignment, some one chunk or less, sources near
    # (in-block chains) and anywhere earlier: the per-wave copies deal full
    # chunks first here, with jobs of very different chunk counts per window
    rng = np.random.default_rng(17)
    blk, ll, ml, sr, lits = [], [], [], [], bytearray()
    total, bs = 0, 1 << 12
    for b in range(256):
        pos, cnt = b * bs, 0
        end = pos + bs
        while pos < end:
            lit = int(rng.integers(0, 12))
            u = rng.random()
            m = int(rng.integers(1, 17)) if u < 0.25 else int(rng.integers(17, 65)) if u < 0.5 \
                else int(rng.integers(65, 401))
            if pos + lit + m <= end and pos + lit >= m:
                lo = 0 if rng.random() < 0.5 else max(0, pos + lit - 2000)
                src = int(rng.integers(lo, pos + lit - m + 1))
                ll.append(lit); ml.append(m); sr.append(src)
                lits += rng.bytes(lit)
                pos += lit + m
            else:
                ll.append(end - pos); ml.append(0); sr.append(0)
                lits += rng.bytes(end - pos)
                pos = end
            cnt += 1
        blk.append(cnt)
        total = end
    c = oracle.pack(total, bs, blk, ll, ml, sr, bytes(lits), tags=False)
    tags, _ = oracle.min_tags(c)
    mlen = np.asarray(ml)
    deferred = mlen[(tags > 0) & (mlen > 0)]
    assert deferred.size > 5000 and deferred.mean() >= 48
    for G in (8, 16, 32):
        check(c, G)


# ------------------------------------------------------------ corruption

def test_corrupt_containers_are_rejected_on_upload():
    x = synth.markov2(1 << 20, seed=13)
    c = oracle.encode(x, 1 << 14, oracle.PRESET_BASE)
    h = oracle.header(c)
    t0 = 64 + 32 * h.n_blocks
    _, ll, ml, src, wave, _ = oracle.tokens(c)
    mi = int(np.nonzero(wave)[0][5])
    bad = []
    b = c.copy(); b[t0 + 16 * mi + 4] ^= 2; bad.append(b)               # length sum
    b = c.copy()
    b[t0 + 16 * mi + 8:t0 + 16 * mi + 13] = np.frombuffer((h.total_len - 1).to_bytes(5, "little"), np.uint8)
    bad.append(b)                                                        # src after dst
    b = c.copy()                                                         # illegal (too small) tag
    sw64 = b[t0 + 16 * mi + 8:t0 + 16 * mi + 16].view(np.uint64)
    sw64[0] = np.uint64(int(sw64[0]) - (1 << 40))
    bad.append(b)
    s = torch.cuda.current_stream()
    for b in bad:
        assert oracle.validate(b) < 0
        with pytest.raises(aclz.AclzError) as e:
            hh = aclz.aclz_upload(b, s)
            aclz.aclz_free(hh)
        assert e.value.code == aclz.ACLZ_E_CORRUPT


def test_output_buffer_checks():
    c = oracle.encode(synth.markov2(10000, seed=1), 1 << 12, oracle.PRESET_BASE)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        small = torch.empty(100, dtype=torch.uint8, device="cuda")
        with pytest.raises(aclz.AclzError) as e:
            aclz.aclz_decode_all(h, small, stream=s)
        assert e.value.code == aclz.ACLZ_E_CAPACITY
        buf = torch.empty(20000, dtype=torch.uint8, device="cuda")
        with pytest.raises(aclz.AclzError) as e:
            aclz.aclz_decode_all(h, buf.data_ptr() + 1, cap=19999, stream=s)
        assert e.value.code == aclz.ACLZ_E_INVAL
        with pytest.raises(aclz.AclzError):
            aclz.aclz_decode_all(h, buf, G=12, stream=s)
    finally:
        aclz.aclz_free(h)


# ------------------------------------------------------------ flatten

def _flatten_case(kind):
    if kind == "fastq_base":
        return oracle.encode(synth.fastq(1 << 20, seed=41), 1 << 12, oracle.PRESET_BASE, chain_depth=16)
    if kind == "markov_base":
        return oracle.encode(synth.markov2(1 << 20, seed=42), 1 << 13, oracle.PRESET_BASE, chain_depth=16)
    if kind == "text_tuned":
        return oracle.encode(synth.wordtext(1 << 20, seed=43, chunk_bytes=1 << 20), 1 << 14, oracle.PRESET_TUNED,
                             chain_depth=16)
    if kind == "tiny_blocks":
        return oracle.encode(synth.fastq(200_000, seed=44), 64, oracle.PRESET_BASE, chain_depth=8)
    L = int(kind[5:])
    sw = synth.copy_sweep(6 << 20, 1 << 15, L, seed=synth.SEED_COPY + 3 * L)
    return oracle.pack_sweep(sw)


@pytest.mark.parametrize("kind", ["fastq_base", "markov_base", "text_tuned", "tiny_blocks", "sweep1024",
                                  "sweep32"])
def test_flatten_decodes_identically(kind):
    c = _flatten_case(kind)
    exp = oracle.decode(c)
    fe = oracle.fnv_chunked(exp)
    before = oracle.header(c).n_waves
    for mode in MODES:
        got, f, info = gpu_decode(c, 32, mode, flatten=True)
        assert np.array_equal(got, exp), mode
        assert f == fe
        assert info["n_waves"] == (2 if before > 1 else before)
    # flatten is idempotent and keeps the container's tags
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        tags = aclz.aclz_tags(h)
        aclz.aclz_flatten(h, s)
        aclz.aclz_flatten(h, s)
        assert np.array_equal(aclz.aclz_tags(h), tags)
        out = torch.empty(len(exp) + 16, dtype=torch.uint8, device="cuda")
        aclz.aclz_decode_all(h, out, G=16, stream=s)
        assert np.array_equal(out[:len(exp)].cpu().numpy(), exp)
    finally:
        aclz.aclz_free(h)


@pytest.mark.parametrize("kind", ["fastq_base", "text_tuned", "tiny_blocks", "sweep1024", "sweep32"])
def test_flatten_upload_without_tags(kind):
    """Upload with ACLZ_UPLOAD_FLATTEN of an untagged container: the 0/1
    tags are exactly 'minimal tag > 0', and every mode decodes the bytes."""
    c = oracle.strip_tags(_flatten_case(kind))
    exp = oracle.decode(c)
    mt, _ = oracle.min_tags(c)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s, flags=aclz.ACLZ_UPLOAD_FLATTEN)
    try:
        assert np.array_equal(aclz.aclz_tags(h), (mt > 0).astype(np.uint32))
        info = aclz.aclz_handle_info(h)
        assert info.n_waves <= 2
        out = torch.empty(len(exp) + 16, dtype=torch.uint8, device="cuda")
        for mode, flags in MODES:
            out.zero_()
            aclz.aclz_decode_all(h, out, mode=mode, flags=flags, stream=s)
            assert aclz.aclz_device_status(h, s) == 0
            assert np.array_equal(out[:len(exp)].cpu().numpy(), exp), (mode, flags)
        # seek is unaffected
        lo, hi = len(exp) // 3, len(exp) // 3 + 100_000
        part = torch.empty(hi - lo + 16, dtype=torch.uint8, device="cuda")
        aclz.aclz_decode_range(h, lo, hi, part, stream=s)
        assert np.array_equal(part[:hi - lo].cpu().numpy(), exp[lo:hi])
    finally:
        aclz.aclz_free(h)


@pytest.mark.parametrize("kind", ["sweep1024", "sweep32", "fastq_base", "text_tuned", "tiny_blocks"])
@pytest.mark.parametrize("rounds", [1, 2])
def test_reshape_cuts_waves_and_decodes_identically(kind, rounds):
    c = _flatten_case(kind)
    exp = oracle.decode(c)
    fe = oracle.fnv_chunked(exp)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        i0 = aclz.aclz_handle_info(h)
        aclz.aclz_reshape(h, rounds, s)
        i1 = aclz.aclz_handle_info(h)
        assert i1.n_tokens >= i0.n_tokens and i1.total_len == i0.total_len
        assert i1.n_waves <= i0.n_waves
        if i0.n_waves > 8:
            assert i1.n_waves < i0.n_waves
        assert aclz.aclz_tags(h).size == i1.n_tokens
        out = torch.empty(len(exp) + 16, dtype=torch.uint8, device="cuda")
        for mode, flags in MODES:
            out.zero_()
            aclz.aclz_decode_all(h, out, mode=mode, flags=flags, stream=s)
            assert aclz.aclz_device_status(h, s) == 0
            assert np.array_equal(out[:len(exp)].cpu().numpy(), exp), (mode, flags)
        assert aclz.aclz_fnv(out, len(exp), stream=s) == fe
        lo, hi = len(exp) // 5, min(len(exp), len(exp) // 5 + 300_000)
        part = torch.empty(hi - lo + 16, dtype=torch.uint8, device="cuda")
        aclz.aclz_decode_range(h, lo, hi, part, stream=s)
        assert np.array_equal(part[:hi - lo].cpu().numpy(), exp[lo:hi])
        # and flattening after reshaping still decodes the bytes
        aclz.aclz_flatten(h, s)
        aclz.aclz_decode_all(h, out, stream=s)
        assert np.array_equal(out[:len(exp)].cpu().numpy(), exp)
        with pytest.raises(aclz.AclzError):
            aclz.aclz_reshape(h, 1, s)
    finally:
        aclz.aclz_free(h)


@pytest.mark.parametrize("kind", ["sweep1024", "fastq_base", "text_tuned"])
def test_export_writes_the_minimal_tags_and_reuploads(kind):
    c = oracle.strip_tags(_flatten_case(kind))
    exp = oracle.decode(c)
    mt, nw = oracle.min_tags(c)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        e = aclz.aclz_export(h)
    finally:
        aclz.aclz_free(h)
    hd = oracle.header(e)
    assert hd.flags == 1 and hd.n_waves == nw
    assert oracle.validate(e) == 0
    assert np.array_equal(oracle.tokens(e)[4], mt)
    assert np.array_equal(oracle.decode(e), exp)
    h = aclz.aclz_upload(e, s)
    try:
        assert np.array_equal(aclz.aclz_tags(h), mt)
        out = torch.empty(len(exp) + 16, dtype=torch.uint8, device="cuda")
        aclz.aclz_decode_all(h, out, stream=s)
        assert np.array_equal(out[:len(exp)].cpu().numpy(), exp)
        # a reshaped handle exports its rewritten tokens, still a legal container
        aclz.aclz_reshape(h, 1, s)
        e2 = aclz.aclz_export(h)
        assert oracle.validate(e2) == 0 and np.array_equal(oracle.decode(e2), exp)
        # flattening keeps the (minimal) tags, so the stream still exports
        aclz.aclz_flatten(h, s)
        e3 = aclz.aclz_export(h)
        assert np.array_equal(e3, e2)
    finally:
        aclz.aclz_free(h)
    # the 0/1 tags of a flattening upload of an untagged container do not
    h = aclz.aclz_upload(c, s, flags=aclz.ACLZ_UPLOAD_FLATTEN)
    try:
        with pytest.raises(aclz.AclzError):
            aclz.aclz_export(h)
    finally:
        aclz.aclz_free(h)


def test_deep_chains_flatten_on_plain_upload():
    """A chain of copies through every block: block b's match copies block
    b - 1's match, so minimal tags run 0 .. n_blocks - 1 and the plain
    schedule's (wave, block) table would pass 2^28 cells; the plain upload
    then builds the flattened schedule, keeps the minimal tags, and decodes
    the bytes."""
    nb, bs = 1 << 17, 64
    total = nb * bs
    blk = np.concatenate([[1], np.ones(nb - 1)]).astype(np.uint32)
    ll = np.full(nb, 48, np.uint32)
    ml = np.full(nb, 16, np.uint32)
    src = (np.arange(nb, dtype=np.uint64) - 1) * bs + 48
    ll[0], ml[0], src[0] = 64, 0, 0
    lits = np.random.default_rng(46).integers(0, 256, int(ll.sum()), dtype=np.uint8)
    c = aclz.aclz_pack(total, bs, (4, 4, 4, 4), blk, ll, ml, src, lits)
    exp = oracle.decode(c)
    mt, nw = oracle.min_tags(c)
    assert nw == nb and (nw - 1) * nb > (1 << 28)
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        assert aclz.aclz_handle_info(h).n_waves == 2
        assert np.array_equal(aclz.aclz_tags(h), mt)
        out = torch.empty(total + 16, dtype=torch.uint8, device="cuda")
        for mode, flags in MODES:
            out.zero_()
            aclz.aclz_decode_all(h, out, mode=mode, flags=flags, stream=s)
            assert aclz.aclz_device_status(h, s) == 0
            assert np.array_equal(out[:total].cpu().numpy(), exp), (mode, flags)
        e = aclz.aclz_export(h)
        assert oracle.header(e).n_waves == nw and np.array_equal(oracle.tokens(e)[4], mt)
    finally:
        aclz.aclz_free(h)


def test_upload_ex_rejects_unknown_flags():
    c = _flatten_case("markov_base")
    with pytest.raises(aclz.AclzError):
        aclz.aclz_upload(c, torch.cuda.current_stream(), flags=6)


# ------------------------------------------------- phase event and plan

@pytest.mark.parametrize("L", [32, 1024])
def test_phase_event_and_plan(L):
    sw = synth.copy_sweep(24 << 20, 1 << 15, L, seed=synth.SEED_COPY + 7 * L)
    c = aclz.aclz_pack(sw.total, sw.block_size, (4, 4, 4, 4), sw.blk_ntok, sw.lit_len, sw.match_len,
                       sw.src, sw.literals)
    exp = oracle.decode(oracle.pack_sweep(sw, tags=False))
    s = torch.cuda.current_stream()
    h = aclz.aclz_upload(c, s)
    try:
        counts = aclz.aclz_wave_counts(h)
        plan, n = aclz.aclz_decode_plan(h, mode=aclz.ACLZ_MODE_WAVES)
        assert plan["mode"] == aclz.ACLZ_MODE_WAVES and n == 1 + int((counts[1:] > 0).sum())
        plan, n = aclz.aclz_decode_plan(h, mode=aclz.ACLZ_MODE_PERSISTENT)
        assert plan["mode"] == aclz.ACLZ_MODE_PERSISTENT and n == 2
        assert plan["flags"] in (aclz.ACLZ_FLAG_STAGED, aclz.ACLZ_FLAG_REGISTERS)
        plan, n = aclz.aclz_decode_plan(h)
        # AUTO: persistent with staging for long deferred matches, waves for short ones
        assert plan["mode"] == (aclz.ACLZ_MODE_PERSISTENT if L == 1024 else aclz.ACLZ_MODE_WAVES)
        with pytest.raises(aclz.AclzError):
            aclz.aclz_decode_plan(h, G=12)
        out = torch.empty(sw.total, dtype=torch.uint8, device="cuda")
        a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        m.record(s)
        out.zero_()
        a.record(s)
        aclz.aclz_decode_all_ev(h, out, m, stream=s)
        b.record(s)
        b.synchronize()
        assert a.elapsed_time(m) > 0 and m.elapsed_time(b) > 0
        assert np.array_equal(out.cpu().numpy(), exp)
    finally:
        aclz.aclz_free(h)


# ------------------------------------------------------------------- FNV

@pytest.mark.parametrize("n", [0, 1, 65535, 65536, 65537, (3 << 20) + 5])
def test_fnv_matches_oracle(n):
    x = np.frombuffer(np.random.default_rng(n).bytes(max(n, 1)), dtype=np.uint8)[:n].copy()
    t = torch.from_numpy(x if n else np.zeros(1, np.uint8)).cuda()
    assert aclz.aclz_fnv(t, n) == oracle.fnv_chunked(x)


# ------------------------------------------------------- full-size case

@pytest.mark.parametrize("L", [1024, 32])
def test_copy_sweep_1gib_full_size(L):
    """1 GiB copy sweep in the benchmark's launch configuration (G = 32,
    32 KiB blocks): every output byte against the oracle, and FNV."""
    sw = synth.copy_sweep(1 << 30, 1 << 15, L, seed=synth.SEED_COPY + L)
    c = aclz.aclz_pack(sw.total, sw.block_size, (4, 4, 4, 4), sw.blk_ntok, sw.lit_len, sw.match_len,
                       sw.src, sw.literals)
    exp = oracle.decode(oracle.pack_sweep(sw, tags=False))
    fe = oracle.fnv_chunked(exp)
    for mode in MODES:
        got, f, info = gpu_decode(c, 32, mode)
        assert np.array_equal(got, exp)
        assert f == fe
    # the benchmark's exact launch: AUTO, 2 CTAs per SM, 4 KiB ranges, phase event
    ev = torch.cuda.Event(enable_timing=True)
    ev.record()
    got, f, info = gpu_decode(c, 32, (aclz.ACLZ_MODE_AUTO, 0), range_bytes=4096, ctas_per_sm=2, phase_event=ev)
    assert np.array_equal(got, exp)
    assert f == fe


# ------------------------------------------------------ failure detection

def test_bounded_wait_times_out_and_the_context_stays_usable():
    """A wait on a completion word that nothing sets gives up after its poll
    limit, reports ACLZ_E_TIMEOUT, and the GPU keeps working (a decode right
    after is exact)."""
    s = torch.cuda.current_stream()
    assert aclz.aclz_selftest_wait(2000, s) == aclz.ACLZ_E_TIMEOUT
    assert aclz.aclz_selftest_wait(0, s) == aclz.ACLZ_E_INVAL
    c = _flatten_case("markov_base")
    got, f, info = gpu_decode(c, 32, PERSIST_STAGED)
    assert np.array_equal(got, oracle.decode(c))
