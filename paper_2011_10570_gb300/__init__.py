"""GB300-native local timestepping (LTS) on 2:1-balanced octrees."""
