"""Each committed ncu summary names the sources it was captured from and their
hash (sha256 of the files' bytes in the listed order, first 16 hex digits);
the hash must match the sources as they are, so that no summary describes a
kernel that has since changed without saying so."""
import hashlib
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1109_3186_gb300", "csrc")


def test_every_profile_hash_matches_its_sources():
    seen = 0
    for fn in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        if not fn.endswith(".md"):
            continue
        txt = open(os.path.join(ROOT, "profiles", fn)).read()
        m = re.search(r"Source hash \(sha256 of ([^,]+), first 16 hex\): `([0-9a-f]{16})`", txt)
        if not m:
            continue
        h = hashlib.sha256()
        for f in (s.strip() for s in m.group(1).split("+")):
            with open(os.path.join(CSRC, f), "rb") as fh:
                h.update(fh.read())
        assert h.hexdigest()[:16] == m.group(2), fn
        seen += 1
    assert seen >= 5
