"""Loader for the worked examples transcribed from the paper (tests/golden/*.json)."""
import json
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        d = json.load(f)
    assert d.get("source"), f"golden fixture {name} lacks its citation"
    return d
