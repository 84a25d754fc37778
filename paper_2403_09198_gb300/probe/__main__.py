from . import run

print(run(), end="")
