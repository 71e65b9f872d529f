"""The checkpoint file's checksum (host code, no GPU): files written through
the library's checkpoint writer, in writes of the sizes sx_save makes
(header, bins, a 4-byte source list, regions), end with a trailer whose
checksum follows its definition (eight FNV-1a streams over the bytes by
offset mod 8, folded with the byte count), and verify; a damaged, truncated
or extended file, a wrong magic or a missing trailer is refused."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MAGIC = b"SXCKPT03"

# the write sizes of sx_save for 42 bins and one source (header, bins,
# source vertices, source rates), then regions of odd sizes
SAVE_LIKE = [208 - 8, 24 * 42, 4, 8, 1_000_003, 77, 5, 4_194_311]


def _fnv_lanes(data: bytes) -> int:
    M, P, B = (1 << 64) - 1, 0x100000001B3, 0xCBF29CE484222325
    lanes = [B] * 8
    for k in range(8):
        h = B
        for byte in data[k::8]:
            h = ((h ^ byte) * P) & M
        lanes[k] = h
    h = B
    for lane in lanes:
        h = ((h ^ lane) * P) & M
    return ((h ^ len(data)) * P) & M


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    exe = tmp_path_factory.mktemp("ckpt") / "ckpt_driver"
    src = os.path.join(ROOT, "tests", "ckpt_driver.cpp")
    inc = os.path.join(ROOT, "paper_0912_4273_gb300", "csrc")
    for flags in (["-fsanitize=address,undefined", "-fno-sanitize-recover=all"], []):
        r = subprocess.run(["g++", "-std=c++17", "-O1", "-g", *flags, "-I", inc, src, "-o", str(exe)],
                           capture_output=True, text=True)
        if r.returncode == 0:
            return exe
    pytest.skip("cannot build the driver: " + r.stderr[-300:])


def _write(driver, path, sizes, seed=1):
    r = subprocess.run([str(driver), str(path), str(seed), *map(str, sizes)], capture_output=True,
                       text=True, timeout=300, env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1"))
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("sizes", [SAVE_LIKE, [1], [7, 1, 1, 1, 13], [8 * 1000], [3] * 50])
def test_trailer_follows_the_definition(driver, tmp_path, sizes):
    path = tmp_path / "a.sxck"
    _write(driver, path, sizes)
    data = path.read_bytes()
    assert data[:8] == MAGIC and len(data) == 8 + sum(sizes) + 16
    assert data[-16:-8] == b"SXCKSUM1"
    assert int.from_bytes(data[-8:], "little") == _fnv_lanes(data[:-16])


def test_library_verifies_and_refuses_damage(driver, tmp_path, libpath):
    from paper_0912_4273_gb300 import simplex as S

    good = tmp_path / "good.sxck"
    _write(driver, good, SAVE_LIKE)
    S.sx_checkpoint_verify(str(good))
    data = good.read_bytes()
    n = len(data)

    def refused(blob, why):
        p = tmp_path / "bad.sxck"
        p.write_bytes(blob)
        with pytest.raises(S.SimplexError) as e:
            S.sx_checkpoint_verify(str(p))
        assert e.value.code == S.SX_EINVAL and why in str(e.value), str(e.value)

    for at in (8, 9, 200, n // 2, n - 17, n - 1):  # one byte changed: body or checksum
        b = bytearray(data)
        b[at] ^= 0x20
        refused(bytes(b), "damaged")
    refused(data[:-1], "no checksum")  # truncated
    refused(data + b"\0", "no checksum")  # extended
    refused(b"SXCKPT01" + data[8:], "not a checkpoint")
    b = bytearray(data)
    b[-16] ^= 1
    refused(bytes(b), "no checksum")
    refused(data[:-16], "no checksum")  # a file without a trailer
    refused(MAGIC + b"\0" * 10, "too short")
    p = tmp_path / "missing.sxck"
    with pytest.raises(S.SimplexError):
        S.sx_checkpoint_verify(str(p))


@pytest.fixture(scope="module")
def libpath():
    from paper_0912_4273_gb300 import build

    return build.build()
